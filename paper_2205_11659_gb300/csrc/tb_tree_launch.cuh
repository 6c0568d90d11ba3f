// tb_tree_launch.cuh -- workspace layout and launch sequences of the tree
// scans, for any monoid: used by the library's C ABI (tb_tree_api.cu) and
// by the public header-only template include/tb_monoid.cuh.  A translation
// unit may define TB_PHASE_MARK(stream) (an event hook before each kernel)
// and TB_WITHHELD_TILE() (the look-back test hook) before including it.
//
// Everything here has internal linkage (an unnamed namespace).  The launch
// functions remember in function-local statics, per device, that a kernel's
// shared-memory limit was raised (tb_device_once.h); with external linkage
// those statics become one object per process (GNU unique symbols), so a
// second shared library built from this header would skip raising the limit
// for its own copy of a kernel and its launch would fail.
#ifndef TB_TREE_LAUNCH_CUH
#define TB_TREE_LAUNCH_CUH

#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "tb.h"
#include "tb_device_once.h"
#include "tb_tree_kernels.cuh"

#ifndef TB_PHASE_MARK
#define TB_PHASE_MARK(stream) ((void)0)
#endif
#ifndef TB_WITHHELD_TILE
#define TB_WITHHELD_TILE() (-1)
#endif

namespace tb {
namespace {
namespace launch {

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

inline TreeLayout tree_layout(int64_t n, bool backward) {
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

inline TreeWs tree_ws(const TreeLayout& L, void* ws, int64_t n, int J) {
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
  w.withhold = TB_WITHHELD_TILE();
  return w;
}

inline bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

// Blocks for a grid-stride kernel over `items`: one per `per_block` items,
// at most 16 per SM of the current device.
inline int grid_for(int items, int per_block) {
  const int g = (items + per_block - 1) / per_block;
  const int sms = current_device_sms();
  const int cap = (sms > 0 ? sms : 1) * 16;
  return g < 1 ? 1 : (g > cap ? cap : g);
}

// Largest dynamic shared memory of one block on this architecture (227 KB).
constexpr size_t kMaxBlockSmem = 227 * 1024;

// Status word, joint depths with the stream checks, tile minima.
inline tb_status prelude(const uint8_t* kind, int64_t n, int J, const TreeLayout& L, void* ws,
                  int32_t* d_status, cudaStream_t s, TreeWs* out) {
  unsigned char* b = static_cast<unsigned char*>(ws);
  TreeWs w = tree_ws(L, ws, n, J);
  w.status = d_status;
  if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess) return TB_ERR_CUDA;
  if (cudaMemsetAsync(b + L.hdr, 0, L.zero_end - L.hdr, s) != cudaSuccess) return TB_ERR_CUDA;
  TB_PHASE_MARK(s);
  k_tdepth<<<L.TE, TNT, 0, s>>>(kind, w, d_status);
  if (cudaGetLastError() != cudaSuccess) return TB_ERR_CUDA;
  if (J > 0) {
    TB_PHASE_MARK(s);
    k_jminmax<<<w.TJ, JNT, 0, s>>>(w);
    if (cudaGetLastError() != cudaSuccess) return TB_ERR_CUDA;
    TB_PHASE_MARK(s);
    k_jmin_tree<<<1, 1024, 0, s>>>(w);
    if (cudaGetLastError() != cudaSuccess) return TB_ERR_CUDA;
  }
  *out = w;
  return TB_OK;
}

template <class M, bool CHAIN>
tb_status launch_jstruct(const TreeWs& w, const void* in, cudaStream_t s) {
  TB_PHASE_MARK(s);
  k_jstruct<M, CHAIN><<<w.TJ, JNT, 0, s>>>(w, in);
  return cudaGetLastError() == cudaSuccess ? TB_OK : TB_ERR_CUDA;
}

// The DOWN scan after its chain input (k_jstruct<M, true> or k_jchain).
template <class M>
tb_status launch_tile_links(const TreeWs& w, int32_t* d_status, cudaStream_t s) {
  TB_PHASE_MARK(s);
  const size_t tsm = down_tiles_smem<M>(w.TJ);
  if (tsm <= kMaxBlockSmem) {
    static std::atomic<unsigned long long> tiles_attr{0};
    if (smem_limit_once(tiles_attr, k_down_tiles<M, true>, kMaxBlockSmem) != cudaSuccess)
      return TB_ERR_CUDA;
    k_down_tiles<M, true><<<1, 1024, tsm, s>>>(w, d_status);
  } else {
    k_down_tiles<M, false><<<1, 1024, 0, s>>>(w, d_status);
  }
  return cudaGetLastError() == cudaSuccess ? TB_OK : TB_ERR_CUDA;
}

template <class M>
tb_status launch_down_tiles(const TreeWs& w, const void* in, void* out, int32_t* d_status,
                            cudaStream_t s) {
  const tb_status st = launch_tile_links<M>(w, d_status, s);
  if (st != TB_OK) return st;
  TB_PHASE_MARK(s);
  constexpr size_t smem = down_tile_smem<M>();
  static std::atomic<unsigned long long> attr_set{0};
  if (smem_limit_once(attr_set, k_down_tile<M>, smem) != cudaSuccess) return TB_ERR_CUDA;
  k_down_tile<M><<<w.TJ, JNT, smem, s>>>(w, in, out);
  if (cudaGetLastError() != cudaSuccess) return TB_ERR_CUDA;
  return TB_OK;
}

template <class M>
tb_status launch_down(const TreeWs& w, const void* in, void* out, int32_t* d_status, cudaStream_t s) {
  tb_status st = launch_jstruct<M, true>(w, in, s);
  if (st != TB_OK) return st;
  return launch_down_tiles<M>(w, in, out, d_status, s);
}

template <class M>
tb_status launch_up_tiles(const TreeWs& w, cudaStream_t s) {
  k_up_tiles<M><<<1, 1024, 0, s>>>(w);
  return cudaGetLastError() == cudaSuccess ? TB_OK : TB_ERR_CUDA;
}

template <class M, class Values, class Finish>
tb_status launch_up(const TreeWs& w, Values values, void* out, Finish fin, cudaStream_t s) {
  TB_PHASE_MARK(s);
  constexpr size_t smem = up_tile_smem<M>();
  static std::atomic<unsigned long long> attr_set{0};
  if (smem_limit_once(attr_set, k_up_tile<M, Values, Finish>, smem) != cudaSuccess) return TB_ERR_CUDA;
  k_up_tile<M, Values, Finish><<<w.TJ, JNT, smem, s>>>(w, values, out, fin);
  if (cudaGetLastError() != cudaSuccess) return TB_ERR_CUDA;
  TB_PHASE_MARK(s);
  const tb_status st = launch_up_tiles<M>(w, s);
  if (st != TB_OK) return st;
  TB_PHASE_MARK(s);
  k_up_cross<M, Values, Finish><<<grid_for(w.TJ * 64, 128), 128, 0, s>>>(w, values, out, fin);
  if (cudaGetLastError() != cudaSuccess) return TB_ERR_CUDA;
  return TB_OK;
}

// The affine adjoint once the joint structure and the tiles' exported
// chains are in the workspace: the tile pass's world folds, one pass per
// tile (world values, adjoint values, their UP fold and the finish), then
// the UP's cross-tile completion.
inline tb_status launch_adjoint(const TreeWs& w, const void* local, const void* grad_world, void* world,
                                void* acc, float* grad_local, int32_t* d_status, cudaStream_t s) {
  tb_status st = launch_tile_links<MonoidAffine>(w, d_status, s);
  if (st != TB_OK) return st;
  TB_PHASE_MARK(s);
  constexpr size_t smem = adjoint_tile_smem();
  static std::atomic<unsigned long long> attr_set{0};
  if (smem_limit_once(attr_set, k_adjoint_tile, smem) != cudaSuccess) return TB_ERR_CUDA;
  const AdjointFinish fin{world, grad_local};
  k_adjoint_tile<<<w.TJ, JNT, smem, s>>>(w, local, grad_world, world, acc, fin);
  if (cudaGetLastError() != cudaSuccess) return TB_ERR_CUDA;
  TB_PHASE_MARK(s);
  st = launch_up_tiles<MonoidAffSum>(w, s);
  if (st != TB_OK) return st;
  TB_PHASE_MARK(s);
  k_up_cross<MonoidAffSum, AdjointValues, AdjointFinish><<<grid_for(w.TJ * 64, 128), 128, 0, s>>>(
      w, AdjointValues{grad_world, world}, acc, fin);
  return cudaGetLastError() == cudaSuccess ? TB_OK : TB_ERR_CUDA;
}

template <class M>
tb_status scan_dir(int dir, const TreeWs& w, const void* in, void* out, int32_t* d_status,
                   cudaStream_t s) {
  if (dir == TB_DOWN) return launch_down<M>(w, in, out, d_status, s);
  tb_status st = launch_jstruct<M, false>(w, nullptr, s);
  if (st != TB_OK) return st;
  return launch_up<M>(w, InputValues<M>{in}, out, NoFinish{}, s);
}

inline tb_status check_common(const uint8_t* kind, int64_t n, int64_t num_joints, void* ws,
                              int32_t* d_status) {
  if (n < 0 || n > kMaxN || d_status == nullptr || !aligned(d_status, 4)) return TB_ERR_INVALID_ARG;
  if (num_joints < 0 || num_joints > n / 2) return TB_ERR_INVALID_ARG;
  if (n > 0 && (kind == nullptr || ws == nullptr || !aligned(kind, 16) || !aligned(ws, 16)))
    return TB_ERR_INVALID_ARG;
  return TB_OK;
}


}  // namespace launch
}  // namespace
}  // namespace tb

#endif  // TB_TREE_LAUNCH_CUH
