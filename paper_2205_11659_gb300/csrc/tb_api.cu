// tb_api.cu -- the C ABI of include/tb.h: argument checks, workspace
// layout and the launch sequence of each operation.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <mutex>

#include "tb.h"
#include "tb_device_once.h"
#include "tb_internal.h"
#include "tb_scene_kernels.cuh"

namespace {

using namespace tb;

constexpr int64_t kMaxN = (int64_t)INT_MAX - TILE;

constexpr size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// Workspace carving shared by tb_workspace_size and the launches.  The tile
// counters (the persistent main pass's ticket) come first so one memset
// clears them.
struct Layout {
  size_t counter, t_a, t_b, t_tot, t_dstart, t_lo, t_ps, t_q, lo_tree, t_link0, t_link1, t_val0,
      t_val1, t_B, t_uall, uall_tree, slice_pos, slice_rel, usuf, upre, cpos, cval, t_seg, t_nseg,
      t_cont, ctx_src, t_boff, t_aoff, t_segb, total;
  int T, P;
  int64_t cap;
};

// Levels of the tiles' union table beyond level 0: floor(log2 T).
constexpr int union_levels(int T) {
  int k = 0;
  while ((2 << k) <= T) ++k;
  return k;
}

constexpr Layout scene_layout(int64_t n, bool has_box) {
  Layout L{};
  const int T = (int)((n + TILE - 1) / TILE);
  const int P = next_pow2(T > 0 ? T : 1);
  L.T = T;
  L.P = P;
  // Slots of the tiles' slices (unmatched opens) and of their closes that
  // match earlier tiles: at most n / 2 of each in a balanced stream (every
  // one pairs with a distinct element of the other side).
  const int64_t cap = n / 2 + 1;
  L.cap = cap;
  const size_t t4 = (size_t)T * 4, t16 = (size_t)T * 16, slots = (size_t)cap;
  size_t o = 0;
  auto take = [&o](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  L.counter = take(16);
  L.t_a = take(t4);
  L.t_b = take(t4);
  L.t_tot = take(t4);
  L.t_dstart = take(t4);
  L.t_lo = take(t4);
  L.t_ps = take(t4);
  L.t_q = take(t4);
  L.lo_tree = take((size_t)2 * P * 4);
  L.slice_pos = take(slots * 4);
  L.cpos = take(slots * 4);
  L.cval = take(slots * 4);
  L.t_seg = take((size_t)T * SEGK * 16);
  L.t_segb = take((size_t)T * SEGK * 4);
  L.t_nseg = take(t4);
  L.t_cont = take((size_t)T * 8);
  L.ctx_src = take(((size_t)cap + T) * 4);
  L.t_boff = take(t4);
  L.t_aoff = take(t4);
  if (has_box) {
    L.t_link0 = take(t4);
    L.t_link1 = take(t4);
    L.t_val0 = take(t16);
    L.t_val1 = take(t16);
    L.t_B = take(t16);
    L.t_uall = take(t16);
    L.uall_tree = take((size_t)union_levels(T) * T * 16);
    L.slice_rel = take(slots * 16);
    L.usuf = take(slots * 16);
    L.upre = take(slots * 16);
  }
  L.total = n > 0 ? o : 0;
  return L;
}

SceneWs scene_ws(const Layout& L, void* ws, bool has_box) {
  unsigned char* b = static_cast<unsigned char*>(ws);
  SceneWs w{};
  w.counter = reinterpret_cast<unsigned*>(b + L.counter);
  w.t_a = reinterpret_cast<int*>(b + L.t_a);
  w.t_b = reinterpret_cast<int*>(b + L.t_b);
  w.t_tot = reinterpret_cast<int*>(b + L.t_tot);
  w.t_dstart = reinterpret_cast<int*>(b + L.t_dstart);
  w.t_lo = reinterpret_cast<int*>(b + L.t_lo);
  w.t_ps = reinterpret_cast<int*>(b + L.t_ps);
  w.t_q = reinterpret_cast<int*>(b + L.t_q);
  w.lo_tree = reinterpret_cast<int*>(b + L.lo_tree);
  w.slice_pos = reinterpret_cast<int*>(b + L.slice_pos);
  w.cpos = reinterpret_cast<int*>(b + L.cpos);
  w.cval = reinterpret_cast<int*>(b + L.cval);
  w.t_seg = reinterpret_cast<int4*>(b + L.t_seg);
  w.t_segb = reinterpret_cast<int*>(b + L.t_segb);
  w.t_nseg = reinterpret_cast<int*>(b + L.t_nseg);
  w.t_cont = reinterpret_cast<int2*>(b + L.t_cont);
  w.ctx_src = reinterpret_cast<int*>(b + L.ctx_src);
  w.t_boff = reinterpret_cast<int*>(b + L.t_boff);
  w.t_aoff = reinterpret_cast<int*>(b + L.t_aoff);
  w.slot_cap = L.cap;
  if (has_box) {
    w.t_link[0] = reinterpret_cast<int*>(b + L.t_link0);
    w.t_link[1] = reinterpret_cast<int*>(b + L.t_link1);
    w.t_val[0] = reinterpret_cast<float4*>(b + L.t_val0);
    w.t_val[1] = reinterpret_cast<float4*>(b + L.t_val1);
    w.t_B = reinterpret_cast<float4*>(b + L.t_B);
    w.t_uall = reinterpret_cast<float4*>(b + L.t_uall);
    w.uall_tree = reinterpret_cast<float4*>(b + L.uall_tree);
    w.slice_rel = reinterpret_cast<float4*>(b + L.slice_rel);
    w.usuf = reinterpret_cast<float4*>(b + L.usuf);
    w.upre = reinterpret_cast<float4*>(b + L.upre);
  }
  w.T = L.T;
  w.P = L.P;
  return w;
}

// Caller-owned events recorded between the kernels of a call.
constexpr int kMaxPhaseEvents = 16;
thread_local cudaEvent_t g_phase_events[kMaxPhaseEvents];
thread_local int g_phase_n = 0;
thread_local int g_phase_next = 0;

// Test hook: an element tile of the following tree-scan calls that never
// publishes its look-back word (-1: none).
thread_local int g_withhold = -1;

inline void phase_mark(cudaStream_t s) {
  if (g_phase_next < g_phase_n) cudaEventRecord(g_phase_events[g_phase_next++], s);
}

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

// Blocks of the main pass that are resident on the current device at once
// (persistent launch), found once per device.
template <bool HAS_BOX, bool BATCHED, bool CLIP>
cudaError_t k3_resident_blocks(int* out) {
  static std::atomic<int> cached[kOnceDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool tracked = dev >= 0 && dev < kOnceDevices;
  if (tracked) {
    const int c = cached[dev].load(std::memory_order_relaxed);
    if (c > 0) {
      *out = c;
      return cudaSuccess;
    }
  }
  const int sms = current_device_sms();
  if (sms <= 0) return cudaErrorInvalidDevice;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k3_tile<HAS_BOX, BATCHED, CLIP>, NT,
                                                    k3_smem_bytes(HAS_BOX));
  if (e != cudaSuccess) return e;
  const int nb = sms * (per_sm > 0 ? per_sm : 1);
  if (tracked) cached[dev].store(nb, std::memory_order_relaxed);
  *out = nb;
  return cudaSuccess;
}

template <bool HAS_BOX, bool BATCHED, bool CLIP = false>
cudaError_t launch_k3(const K3Args& a, int T, cudaStream_t s) {
  if (TB_MATCHER == 1 && !HAS_BOX && !BATCHED) {
    // the binary-search form of the matching-only pass (an autotuner candidate)
    k3_search<<<T, NT, k3s_smem_bytes(), s>>>(a);
    return cudaGetLastError();
  }
  constexpr int smem = k3_smem_bytes(HAS_BOX);
  static std::atomic<unsigned long long> attr_set{0};
  cudaError_t e = smem_limit_once(attr_set, k3_tile<HAS_BOX, BATCHED, CLIP>, smem);
  if (e != cudaSuccess) return e;
  int grid = T;
  if (PERSIST) {
    int nb = 0;
    e = k3_resident_blocks<HAS_BOX, BATCHED, CLIP>(&nb);
    if (e != cudaSuccess) return e;
    grid = T < nb ? T : nb;
  }
  k3_tile<HAS_BOX, BATCHED, CLIP><<<grid, NT, smem, s>>>(a);
  return cudaGetLastError();
}

// Blocks of k2_jump that are resident on the current device at once (the
// most a cooperative launch may use), found once per device.
cudaError_t k2_jump_max_blocks(int* out) {
  static std::atomic<int> cached[kOnceDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool tracked = dev >= 0 && dev < kOnceDevices;
  if (tracked) {
    const int c = cached[dev].load(std::memory_order_relaxed);
    if (c > 0) {
      *out = c;
      return cudaSuccess;
    }
  }
  const int sms = current_device_sms();
  if (sms <= 0) return cudaErrorInvalidDevice;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k2_jump, NTJ, 0);
  if (e != cudaSuccess) return e;
  const int nb = sms * (per_sm > 0 ? per_sm : 1);
  if (tracked) cached[dev].store(nb, std::memory_order_relaxed);
  *out = nb;
  return cudaSuccess;
}

// The same for k4_union_table.
cudaError_t k4_table_max_blocks(int* out) {
  static std::atomic<int> cached[kOnceDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool tracked = dev >= 0 && dev < kOnceDevices;
  if (tracked) {
    const int c = cached[dev].load(std::memory_order_relaxed);
    if (c > 0) {
      *out = c;
      return cudaSuccess;
    }
  }
  const int sms = current_device_sms();
  if (sms <= 0) return cudaErrorInvalidDevice;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k4_union_table, NTU, 0);
  if (e != cudaSuccess) return e;
  const int nb = sms * (per_sm > 0 ? per_sm : 1);
  if (tracked) cached[dev].store(nb, std::memory_order_relaxed);
  *out = nb;
  return cudaSuccess;
}

cudaError_t launch_union_table(const SceneWs& w, cudaStream_t s) {
  int levels = union_levels(w.T) + 1;  // level 0 is t_uall
  if (levels < 2) return cudaSuccess;  // one tile: nothing to build
  int maxb = 0;
  cudaError_t e = k4_table_max_blocks(&maxb);
  if (e != cudaSuccess) return e;
  const int want = (w.T + NTU - 1) / NTU;
  const int blocks = want < maxb ? want : maxb;
  SceneWs wa = w;
  void* args[] = {&wa, &levels};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(&k4_union_table), dim3(blocks),
                                     dim3(NTU), args, 0, s);
}

template <bool HAS_BOX>
cudaError_t launch_k2(const SceneWs& w, cudaStream_t s) {
  const int g = (w.T + NTR - 1) / NTR;
  k2_links<<<g, NTR, 0, s>>>(w);
  k2_segments<HAS_BOX><<<g, NTR, 0, s>>>(w);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !HAS_BOX) return e;
  int maxb = 0;
  e = k2_jump_max_blocks(&maxb);
  if (e != cudaSuccess) return e;
  const int want = (w.T + NTJ - 1) / NTJ;
  const int blocks = want < maxb ? want : maxb;
  int rounds = 1;
  while ((1 << (rounds - 1)) < w.T) ++rounds;  // ceil(log2 T) + 1
  SceneWs wa = w;
  void* args[] = {&wa, &rounds};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(&k2_jump), dim3(blocks),
                                     dim3(NTJ), args, 0, s);
}

// The whole matching / bounding-box pass over one stream (a single scene
// or a batch laid end to end).
template <bool HAS_BOX>
tb_status run_scene(const uint8_t* kind, const float* box, int64_t n, int32_t* parent,
                    int32_t* match, float* box_out, const int64_t* offsets, int64_t num_scenes,
                    void* ws, size_t ws_bytes, int32_t* d_status, void* stream,
                    float* clip_out = nullptr) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n < 0 || n > kMaxN || d_status == nullptr) return TB_ERR_INVALID_ARG;
  if (!aligned(d_status, 4)) return TB_ERR_INVALID_ARG;
  if (n > 0) {
    if (kind == nullptr || ws == nullptr) return TB_ERR_INVALID_ARG;
    if (!aligned(kind, 16) || !aligned(ws, 16)) return TB_ERR_INVALID_ARG;
    if (HAS_BOX && (box == nullptr || box_out == nullptr || !aligned(box, 16) ||
                    !aligned(box_out, 16)))
      return TB_ERR_INVALID_ARG;
    if (!HAS_BOX && (parent == nullptr || match == nullptr)) return TB_ERR_INVALID_ARG;
    if ((parent && !aligned(parent, 4)) || (match && !aligned(match, 4))) return TB_ERR_INVALID_ARG;
    if (clip_out && !aligned(clip_out, 16)) return TB_ERR_INVALID_ARG;
    if (offsets != nullptr && (num_scenes < 1 || num_scenes > INT_MAX - 1 || !aligned(offsets, 8)))
      return TB_ERR_INVALID_ARG;
  }
  const Layout L = scene_layout(n, HAS_BOX);
  if (n > 0 && ws_bytes < L.total) return TB_ERR_WORKSPACE;
  if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess) return TB_ERR_CUDA;
  if (n == 0) return TB_OK;

  SceneWs w = scene_ws(L, ws, HAS_BOX);
  w.status = d_status;
  if (cudaMemsetAsync(ws, 0, L.t_a, s) != cudaSuccess) return TB_ERR_CUDA;

  phase_mark(s);
  K1Args a1{kind, reinterpret_cast<const float4*>(box), (int)n, w, d_status};
  k1_tile_summary<HAS_BOX><<<L.T, NT, 0, s>>>(a1);
  k1_tile_prefix<<<1, NT2, 0, s>>>(w, d_status);
  if (cudaGetLastError() != cudaSuccess) return TB_ERR_CUDA;
  phase_mark(s);
  if (launch_k2<HAS_BOX>(w, s) != cudaSuccess) return TB_ERR_CUDA;

  phase_mark(s);
  const int vec_out = (!parent || aligned(parent, 16)) && (!match || aligned(match, 16));
  K3Args a3{kind, reinterpret_cast<const float4*>(box), (int)n, parent, match,
            reinterpret_cast<float4*>(box_out), offsets, (int)num_scenes, vec_out, w, d_status,
            reinterpret_cast<float4*>(clip_out)};
  cudaError_t e;
  if (HAS_BOX && clip_out)
    e = offsets ? launch_k3<HAS_BOX, true, true>(a3, L.T, s) : launch_k3<HAS_BOX, false, true>(a3, L.T, s);
  else
    e = offsets ? launch_k3<HAS_BOX, true>(a3, L.T, s) : launch_k3<HAS_BOX, false>(a3, L.T, s);
  if (e != cudaSuccess) return TB_ERR_CUDA;
  phase_mark(s);
  if (HAS_BOX) {
    if (launch_union_table(w, s) != cudaSuccess) return TB_ERR_CUDA;
  }
  K4Args a4{reinterpret_cast<float4*>(box_out), match, w};
  k4_cross_tile_unions<HAS_BOX><<<L.T, NT, 0, s>>>(a4);
  if (cudaGetLastError() != cudaSuccess) return TB_ERR_CUDA;
  phase_mark(s);
  return TB_OK;
}

}  // namespace

extern "C" {

size_t tb_workspace_size(int op, int64_t n, int64_t num_scenes) {
  (void)num_scenes;
  if (n <= 0 || n > kMaxN) return 0;
  switch (op) {
    case TB_OP_MATCH_PARENS:
      return scene_layout(n, false).total;
    case TB_OP_BBOXES:
    case TB_OP_BBOXES_BATCHED:
      return scene_layout(n, true).total;
    case TB_OP_TREE_SCAN:
    case TB_OP_TREE_BACKWARD:
      return tb_internal::tree_ws_bytes(op, n);
    case TB_OP_OPEN_POSITIONS:
      return tb_internal::open_ws_bytes(n);
    default:
      return 0;
  }
}

tb_status tb_match_parens(const uint8_t* kind, int64_t n, int32_t* parent, int32_t* match, void* ws,
                          size_t ws_bytes, int32_t* d_status, void* stream) {
  g_phase_next = 0;
  return run_scene<false>(kind, nullptr, n, parent, match, nullptr, nullptr, 0, ws, ws_bytes,
                          d_status, stream);
}

tb_status tb_bboxes(const uint8_t* kind, const float* box, int64_t n, int32_t* parent,
                    int32_t* match, float* box_out, void* ws, size_t ws_bytes, int32_t* d_status,
                    void* stream) {
  g_phase_next = 0;
  return run_scene<true>(kind, box, n, parent, match, box_out, nullptr, 0, ws, ws_bytes, d_status,
                         stream);
}

tb_status tb_bboxes_batched(const uint8_t* kind, const float* box, const int64_t* offsets,
                            int64_t num_scenes, int64_t n_total, int32_t* parent, int32_t* match,
                            float* box_out, void* ws, size_t ws_bytes, int32_t* d_status,
                            void* stream) {
  if (offsets == nullptr || num_scenes < 1) return TB_ERR_INVALID_ARG;
  g_phase_next = 0;
  return run_scene<true>(kind, box, n_total, parent, match, box_out, offsets, num_scenes, ws,
                         ws_bytes, d_status, stream);
}

tb_status tb_bboxes_clip(const uint8_t* kind, const float* box, const int64_t* offsets,
                         int64_t num_scenes, int64_t n, int32_t* parent, int32_t* match,
                         float* box_out, float* clip_out, void* ws, size_t ws_bytes,
                         int32_t* d_status, void* stream) {
  if (clip_out == nullptr && n > 0) return TB_ERR_INVALID_ARG;
  if (offsets != nullptr && num_scenes < 1) return TB_ERR_INVALID_ARG;
  g_phase_next = 0;
  return run_scene<true>(kind, box, n, parent, match, box_out, offsets,
                         offsets ? num_scenes : 0, ws, ws_bytes, d_status, stream, clip_out);
}

tb_status tb_set_phase_events(void* const* events, int num_events) {
  if (events == nullptr) {
    g_phase_n = 0;
    return TB_OK;
  }
  if (num_events < 1 || num_events > kMaxPhaseEvents) return TB_ERR_INVALID_ARG;
  for (int i = 0; i < num_events; ++i)
    if (events[i] == nullptr) return TB_ERR_INVALID_ARG;
  for (int i = 0; i < num_events; ++i) g_phase_events[i] = static_cast<cudaEvent_t>(events[i]);
  g_phase_n = num_events;
  return TB_OK;
}

const char* tb_version(void) { return "treebox-gb300 0.1 (sm_103a)"; }

tb_status tb_debug_withhold_tile(int tile) {
  if (tile < -1) return TB_ERR_INVALID_ARG;
  g_withhold = tile;
  return TB_OK;
}

}  // extern "C"

namespace tb_internal {

void phase_reset() { g_phase_next = 0; }
void phase_mark(cudaStream_t s) { ::phase_mark(s); }
int withheld_tile() { return g_withhold; }

}  // namespace tb_internal

// ---------------------------------------------------------------------------
// Allocation-free variant of tb_bboxes.  Its scratch is this file-scope
// device array, so a caller needs no workspace at all.  The array is part of
// the module image: every GPU that loads the library holds it until exit.
namespace {

constexpr size_t kStaticWsBytes = (size_t)5 << 20;  // 5 MiB
static_assert(scene_layout(TB_STATIC_WS_MAX_N, true).total <= kStaticWsBytes,
              "the static scratch must hold the workspace of TB_STATIC_WS_MAX_N elements");

__device__ __align__(256) unsigned char g_tb_static_ws[kStaticWsBytes];

// Device address of g_tb_static_ws per device ordinal, looked up once with that
// device current (host code cannot use the symbol itself as an address).
constexpr int kMaxDevices = 64;
void* g_static_ws_ptr[kMaxDevices] = {};
std::mutex g_static_ws_mu;

tb_status static_ws_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TB_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_static_ws_mu);
  if (g_static_ws_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_tb_static_ws) != cudaSuccess || p == nullptr) return TB_ERR_CUDA;
    g_static_ws_ptr[dev] = p;
  }
  *out = g_static_ws_ptr[dev];
  return TB_OK;
}

}  // namespace

extern "C" {

tb_status tb_bboxes_static_ws(const uint8_t* kind, const float* box, int64_t n, int32_t* parent,
                              int32_t* match, float* box_out, int32_t* d_status, void* stream) {
  if (n < 0) return TB_ERR_INVALID_ARG;
  if (n > TB_STATIC_WS_MAX_N) return TB_ERR_WORKSPACE;
  const Layout L = scene_layout(n, true);
  if (L.total > kStaticWsBytes) return TB_ERR_WORKSPACE;
  void* ws = nullptr;
  const tb_status st = static_ws_for_current_device(&ws);
  if (st != TB_OK) return st;
  // run_scene clears the tile counters of the scratch on every call;
  // everything else in it is written before it is read.
  g_phase_next = 0;
  return run_scene<true>(kind, box, n, parent, match, box_out, nullptr, 0, ws, kStaticWsBytes,
                         d_status, stream);
}

}  // extern "C"
