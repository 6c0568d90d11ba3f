// tb_tree_api.cu -- the tree scans of include/tb.h: argument checks,
// workspace layout and launch sequences.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "tb.h"
#include "tb_internal.h"
#include "tb_tree_kernels.cuh"

namespace {

using namespace tb;

constexpr int64_t kMaxN = (int64_t)INT_MAX - TTILE;
constexpr size_t kValBytes = sizeof(Aff);  // the widest monoid value

constexpr size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// What must start at zero is adjacent so one memset clears it: the
// structure header (a call that rebuilds the joint structure invalidates it
// first), the look-back words and the two counters.
struct TreeLayout {
  size_t lb, counter, xcount, hdr, zero_end, jdepth, premin, sufmin, jparent, jend, g_tree, relT, t_base,
      t_link0, t_link1, t_val0, t_val1, t_world, ctree, t_tree, xlist, world, acc, total;
  int TE, TJ, PJ, Jmax;
};

TreeLayout tree_layout(int64_t n, bool backward) {
  TreeLayout L{};
  const int TE = (int)((n + TTILE - 1) / TTILE);
  const int Jmax = (int)(n / 2);
  const int TJ = (Jmax + JT - 1) / JT;
  const int PJ = next_pow2(TJ > 0 ? TJ : 1);
  L.TE = TE;
  L.TJ = TJ;
  L.PJ = PJ;
  L.Jmax = Jmax;
  size_t o = 0;
  auto take = [&o](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  L.hdr = 0;  // at a fixed place, whatever n: a later call reads it first
  o += 16;
  L.lb = o;
  o += (size_t)TE * 8;
  L.counter = o;
  o += 4;
  L.xcount = o;
  o += 4;
  L.zero_end = o;
  o = align_up(o);
  const size_t J4 = (size_t)Jmax * 4, JV = (size_t)Jmax * kValBytes;
  L.jdepth = take(J4);
  L.premin = take(J4);
  L.sufmin = take(J4);
  L.jparent = take(J4);
  L.jend = take(J4);
  L.g_tree = take((size_t)2 * PJ * 4);
  L.relT = take(JV);
  L.t_base = take((size_t)TJ * 4);
  L.t_link0 = take((size_t)TJ * 4);
  L.t_link1 = take((size_t)TJ * 4);
  L.t_val0 = take((size_t)TJ * kValBytes);
  L.t_val1 = take((size_t)TJ * kValBytes);
  L.t_world = take((size_t)TJ * kValBytes);
  L.ctree = take((size_t)TJ * 2 * NCH * kValBytes);
  L.t_tree = take((size_t)2 * PJ * kValBytes);
  L.xlist = take(J4);
  if (backward) {
    L.world = take(JV);
    L.acc = take(JV);
  }
  L.total = n > 0 ? o : 0;
  return L;
}

TreeWs tree_ws(const TreeLayout& L, void* ws, int64_t n, int J) {
  unsigned char* b = static_cast<unsigned char*>(ws);
  TreeWs w{};
  w.lb = reinterpret_cast<unsigned long long*>(b + L.lb);
  w.counter = reinterpret_cast<unsigned*>(b + L.counter);
  w.xcount = reinterpret_cast<unsigned*>(b + L.xcount);
  w.hdr = reinterpret_cast<int*>(b + L.hdr);
  w.jdepth = reinterpret_cast<int*>(b + L.jdepth);
  w.premin = reinterpret_cast<int*>(b + L.premin);
  w.sufmin = reinterpret_cast<int*>(b + L.sufmin);
  w.jparent = reinterpret_cast<int*>(b + L.jparent);
  w.jend = reinterpret_cast<int*>(b + L.jend);
  w.g_tree = reinterpret_cast<int*>(b + L.g_tree);
  w.relT = b + L.relT;
  w.t_base = reinterpret_cast<int*>(b + L.t_base);
  w.t_link[0] = reinterpret_cast<int*>(b + L.t_link0);
  w.t_link[1] = reinterpret_cast<int*>(b + L.t_link1);
  w.t_val[0] = b + L.t_val0;
  w.t_val[1] = b + L.t_val1;
  w.t_world = b + L.t_world;
  w.ctree = b + L.ctree;
  w.t_tree = b + L.t_tree;
  w.xlist = reinterpret_cast<int*>(b + L.xlist);
  w.n = (int)n;
  w.J = J;
  w.TE = L.TE;
  w.TJ = (J + JT - 1) / JT;
  w.PJ = next_pow2(w.TJ > 0 ? w.TJ : 1);
  w.withhold = tb_internal::withheld_tile();
  return w;
}

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

int grid_for(int items, int per_block) {
  const int g = (items + per_block - 1) / per_block;
  return g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g);
}

// Largest dynamic shared memory of one block on this architecture (227 KB).
constexpr size_t kMaxBlockSmem = 227 * 1024;

template <class K>
cudaError_t allow_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Status word, joint depths with the stream checks, tile minima.
tb_status prelude(const uint8_t* kind, int64_t n, int J, const TreeLayout& L, void* ws,
                  int32_t* d_status, cudaStream_t s, TreeWs* out) {
  unsigned char* b = static_cast<unsigned char*>(ws);
  TreeWs w = tree_ws(L, ws, n, J);
  w.status = d_status;
  if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess) return TB_ERR_CUDA;
  if (cudaMemsetAsync(b + L.hdr, 0, L.zero_end - L.hdr, s) != cudaSuccess) return TB_ERR_CUDA;
  tb_internal::phase_mark(s);
  k_tdepth<<<L.TE, TNT, 0, s>>>(kind, w, d_status);
  if (cudaGetLastError() != cudaSuccess) return TB_ERR_CUDA;
  if (J > 0) {
    tb_internal::phase_mark(s);
    k_jminmax<<<w.TJ, TNT, 0, s>>>(w);
    if (cudaGetLastError() != cudaSuccess) return TB_ERR_CUDA;
    tb_internal::phase_mark(s);
    k_jmin_tree<<<1, 1024, 0, s>>>(w);
    if (cudaGetLastError() != cudaSuccess) return TB_ERR_CUDA;
  }
  *out = w;
  return TB_OK;
}

template <class M, bool CHAIN>
tb_status launch_jstruct(const TreeWs& w, const void* in, cudaStream_t s) {
  tb_internal::phase_mark(s);
  k_jstruct<M, CHAIN><<<w.TJ, TNT, 0, s>>>(w, in);
  return cudaGetLastError() == cudaSuccess ? TB_OK : TB_ERR_CUDA;
}

// The DOWN scan after its chain input (k_jstruct<M, true> or k_jchain).
template <class M>
tb_status launch_down_tiles(const TreeWs& w, const void* in, void* out, int32_t* d_status,
                            cudaStream_t s) {
  tb_internal::phase_mark(s);
  const size_t tsm = down_tiles_smem<M>(w.TJ);
  if (tsm <= kMaxBlockSmem) {
    static bool tiles_attr = false;
    if (!tiles_attr) {
      if (allow_smem(k_down_tiles<M, true>, kMaxBlockSmem) != cudaSuccess) return TB_ERR_CUDA;
      tiles_attr = true;
    }
    k_down_tiles<M, true><<<1, 1024, tsm, s>>>(w, d_status);
  } else {
    k_down_tiles<M, false><<<1, 1024, 0, s>>>(w, d_status);
  }
  if (cudaGetLastError() != cudaSuccess) return TB_ERR_CUDA;
  tb_internal::phase_mark(s);
  constexpr size_t smem = down_tile_smem<M>();
  static bool attr_set = false;
  if (!attr_set) {
    if (allow_smem(k_down_tile<M>, smem) != cudaSuccess) return TB_ERR_CUDA;
    attr_set = true;
  }
  k_down_tile<M><<<w.TJ, TNT, smem, s>>>(w, in, out);
  if (cudaGetLastError() != cudaSuccess) return TB_ERR_CUDA;
  return TB_OK;
}

template <class M>
tb_status launch_down(const TreeWs& w, const void* in, void* out, int32_t* d_status, cudaStream_t s) {
  tb_status st = launch_jstruct<M, true>(w, in, s);
  if (st != TB_OK) return st;
  return launch_down_tiles<M>(w, in, out, d_status, s);
}

template <class M, class Values, class Finish>
tb_status launch_up(const TreeWs& w, Values values, void* out, Finish fin, cudaStream_t s) {
  tb_internal::phase_mark(s);
  constexpr size_t smem = up_tile_smem<M>();
  static bool attr_set = false;
  if (!attr_set) {
    if (allow_smem(k_up_tile<M, Values, Finish>, smem) != cudaSuccess) return TB_ERR_CUDA;
    attr_set = true;
  }
  k_up_tile<M, Values, Finish><<<w.TJ, TNT, smem, s>>>(w, values, out, fin);
  if (cudaGetLastError() != cudaSuccess) return TB_ERR_CUDA;
  tb_internal::phase_mark(s);
  k_up_tiles<M><<<1, 1024, 0, s>>>(w);
  if (cudaGetLastError() != cudaSuccess) return TB_ERR_CUDA;
  tb_internal::phase_mark(s);
  k_up_cross<M, Values, Finish><<<grid_for(w.TJ * 64, 256), 256, 0, s>>>(w, values, out, fin);
  if (cudaGetLastError() != cudaSuccess) return TB_ERR_CUDA;
  return TB_OK;
}

template <class M>
tb_status scan_dir(int dir, const TreeWs& w, const void* in, void* out, int32_t* d_status,
                   cudaStream_t s) {
  if (dir == TB_DOWN) return launch_down<M>(w, in, out, d_status, s);
  tb_status st = launch_jstruct<M, false>(w, nullptr, s);
  if (st != TB_OK) return st;
  return launch_up<M>(w, InputValues<M>{in}, out, NoFinish{}, s);
}

tb_status check_common(const uint8_t* kind, int64_t n, int64_t num_joints, void* ws,
                       int32_t* d_status) {
  if (n < 0 || n > kMaxN || d_status == nullptr || !aligned(d_status, 4)) return TB_ERR_INVALID_ARG;
  if (num_joints < 0 || num_joints > n / 2) return TB_ERR_INVALID_ARG;
  if (n > 0 && (kind == nullptr || ws == nullptr || !aligned(kind, 16) || !aligned(ws, 16)))
    return TB_ERR_INVALID_ARG;
  return TB_OK;
}

}  // namespace

namespace tb_internal {
size_t tree_ws_bytes(int op, int64_t n) {
  if (n <= 0 || n > kMaxN) return 0;
  return tree_layout(n, op == TB_OP_TREE_BACKWARD).total;
}
}  // namespace tb_internal

extern "C" {

tb_status tb_tree_scan(int monoid, int dir, const uint8_t* kind, int64_t n, int64_t num_joints,
                       const void* in, void* out, void* ws, size_t ws_bytes, int32_t* d_status,
                       void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tb_internal::phase_reset();
  if (monoid < TB_MONOID_BBOX_ISECT || monoid > TB_MONOID_AFFINE3X4_F32) return TB_ERR_INVALID_ARG;
  if (dir != TB_DOWN && dir != TB_UP) return TB_ERR_INVALID_ARG;
  tb_status st = check_common(kind, n, num_joints, ws, d_status);
  if (st != TB_OK) return st;
  if (num_joints > 0) {
    if (in == nullptr || out == nullptr || !aligned(in, 16) || !aligned(out, 16) || in == out)
      return TB_ERR_INVALID_ARG;
  }
  const TreeLayout L = tree_layout(n, false);
  if (n > 0 && ws_bytes < L.total) return TB_ERR_WORKSPACE;
  if (n == 0) return cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) == cudaSuccess ? TB_OK : TB_ERR_CUDA;
  TreeWs w;
  st = prelude(kind, n, (int)num_joints, L, ws, d_status, s, &w);
  if (st != TB_OK || num_joints == 0) {
    if (st == TB_OK) tb_internal::phase_mark(s);
    return st;
  }
  switch (monoid) {
    case TB_MONOID_BBOX_ISECT:
      st = scan_dir<MonoidIsect>(dir, w, in, out, d_status, s);
      break;
    case TB_MONOID_BBOX_UNION:
      st = scan_dir<MonoidUnion>(dir, w, in, out, d_status, s);
      break;
    case TB_MONOID_ADD_I32:
      st = scan_dir<MonoidAddI32>(dir, w, in, out, d_status, s);
      break;
    default:
      st = scan_dir<MonoidAffine>(dir, w, in, out, d_status, s);
      break;
  }
  if (st == TB_OK) tb_internal::phase_mark(s);
  return st;
}

tb_status tb_tree_scan_affine_backward(const uint8_t* kind, int64_t n, int64_t num_joints,
                                       const float* local, const float* grad_world,
                                       float* grad_local, void* ws, size_t ws_bytes,
                                       int32_t* d_status, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tb_internal::phase_reset();
  tb_status st = check_common(kind, n, num_joints, ws, d_status);
  if (st != TB_OK) return st;
  if (num_joints > 0) {
    if (local == nullptr || grad_world == nullptr || grad_local == nullptr || !aligned(local, 16) ||
        !aligned(grad_world, 16) || !aligned(grad_local, 16) || grad_local == local ||
        grad_local == grad_world)
      return TB_ERR_INVALID_ARG;
  }
  const TreeLayout L = tree_layout(n, true);
  if (n > 0 && ws_bytes < L.total) return TB_ERR_WORKSPACE;
  if (n == 0) return cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) == cudaSuccess ? TB_OK : TB_ERR_CUDA;
  TreeWs w;
  st = prelude(kind, n, (int)num_joints, L, ws, d_status, s, &w);
  if (st != TB_OK || num_joints == 0) {
    if (st == TB_OK) tb_internal::phase_mark(s);
    return st;
  }
  unsigned char* b = static_cast<unsigned char*>(ws);
  void* world = b + L.world;
  void* acc = b + L.acc;
  st = launch_down<MonoidAffine>(w, local, world, d_status, s);
  if (st != TB_OK) return st;
  st = launch_up<MonoidAffSum>(w, AdjointValues{grad_world, world}, acc,
                               AdjointFinish{world, grad_local}, s);
  if (st != TB_OK) return st;
  tb_internal::phase_mark(s);
  return TB_OK;
}

tb_status tb_tree_scan_affine_backward_reuse(const uint8_t* kind, int64_t n, int64_t num_joints,
                                             const float* local, const float* grad_world,
                                             float* grad_local, void* ws, size_t ws_bytes,
                                             int32_t* d_status, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tb_internal::phase_reset();
  tb_status st = check_common(kind, n, num_joints, ws, d_status);
  if (st != TB_OK) return st;
  if (num_joints > 0) {
    if (local == nullptr || grad_world == nullptr || grad_local == nullptr || !aligned(local, 16) ||
        !aligned(grad_world, 16) || !aligned(grad_local, 16) || grad_local == local ||
        grad_local == grad_world)
      return TB_ERR_INVALID_ARG;
  }
  const TreeLayout L = tree_layout(n, true);
  if (n > 0 && ws_bytes < L.total) return TB_ERR_WORKSPACE;
  if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess) return TB_ERR_CUDA;
  if (n == 0 || num_joints == 0) return TB_OK;
  unsigned char* b = static_cast<unsigned char*>(ws);
  TreeWs w = tree_ws(L, ws, n, (int)num_joints);
  w.status = d_status;
  // only the subtree-list counter restarts; the structure and its header stay
  if (cudaMemsetAsync(b + L.xcount, 0, 4, s) != cudaSuccess) return TB_ERR_CUDA;
  void* world = b + L.world;
  void* acc = b + L.acc;
  tb_internal::phase_mark(s);
  k_jchain<MonoidAffine><<<w.TJ, TNT, 0, s>>>(w, local, d_status);
  if (cudaGetLastError() != cudaSuccess) return TB_ERR_CUDA;
  st = launch_down_tiles<MonoidAffine>(w, local, world, d_status, s);
  if (st != TB_OK) return st;
  st = launch_up<MonoidAffSum>(w, AdjointValues{grad_world, world}, acc,
                               AdjointFinish{world, grad_local}, s);
  if (st != TB_OK) return st;
  tb_internal::phase_mark(s);
  return TB_OK;
}

}  // extern "C"
