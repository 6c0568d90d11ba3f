// tb_core.cuh -- shared pieces of the scene kernels: tile geometry, the box
// algebra, block-wide scans, the min/union segment trees and the
// device-side view of the workspace.
#ifndef TB_CORE_CUH
#define TB_CORE_CUH

#include <cstdint>
#include <climits>
#include <cmath>
#include <cstring>

#include "tb_prims.cuh"

namespace tb {

// ---------------------------------------------------------------- geometry
// A tile is TILE consecutive elements handled by one block of NT threads;
// thread j owns the KPT consecutive elements [j*KPT, j*KPT + KPT) of the
// tile (its "chunk").
// The shape is a build parameter (TB_NT threads per block, TB_KPT elements
// per thread), chosen among a few candidates by the project's autotuner;
// 256 x 16 when not given.
#ifndef TB_NT
#define TB_NT 256
#endif
#ifndef TB_KPT
#define TB_KPT 16
#endif
// TB_PERSIST: the main tile pass runs as persistent blocks (as many as fit
// on the device at once, each taking tiles in turn) instead of one block per
// tile; also chosen by the autotuner.
#ifndef TB_PERSIST
#define TB_PERSIST 0
#endif
constexpr int NT = TB_NT;
constexpr int KPT = TB_KPT;
constexpr bool PERSIST = TB_PERSIST != 0;
constexpr int TILE = NT * KPT;
constexpr int NW = NT / 32;
static_assert(NT == 64 || NT == 128 || NT == 256 || NT == 512, "block size must be 64, 128, 256 or 512");
static_assert(KPT == 8 || KPT == 12 || KPT == 16, "elements per thread must be 8, 12 or 16");

// Element kinds; K_PAD marks positions past the end of the stream.
constexpr int K_LEAF = 0, K_CLIP = 1, K_BLEND = 2, K_CLOSE = 3, K_PAD = 4;

// Status codes (same values as tb_status in tb.h).
constexpr int ST_OK = 0, ST_UNBALANCED = 2, ST_BAD_KIND = 3, ST_TIMEOUT = 5, ST_BOUNDS = 7;

// TB_DEBUG: a build whose kernels check the data-dependent indices of their
// memory accesses (indices read from the workspace or derived from the
// input) before using them.  A failed check records ST_BOUNDS in the status
// word and the access is skipped -- no trap, the context stays usable.  In
// normal builds in_range() is the constant true and the checks vanish.
#ifndef TB_DEBUG
#define TB_DEBUG 0
#endif
__device__ __forceinline__ bool in_range(long long i, long long lo, long long hi, const int* status) {
  if (!TB_DEBUG) return true;
  if (i >= lo && i < hi) return true;
  atomic_cas_i32(const_cast<int*>(status), ST_OK, ST_BOUNDS);
  return false;
}

// Staged boxes are padded by one float4 per chunk so that the 32 lanes of a
// warp, each reading element i of its own chunk, hit distinct banks.
constexpr int BOX_SMEM_LEN = TILE + TILE / KPT;
__host__ __device__ __forceinline__ int box_slot(int p) { return p + p / KPT; }

// Bounded waits: a poll loop gives up after this many iterations (about a
// second with the backoff of poll_backoff) and reports ST_TIMEOUT.
constexpr unsigned SPIN_LIMIT = 1u << 20;

__host__ __device__ __forceinline__ constexpr int kind_delta(int k) {
  return k == K_CLOSE ? -1 : ((k == K_CLIP || k == K_BLEND) ? 1 : 0);
}
__host__ __device__ __forceinline__ constexpr bool kind_open(int k) { return k == K_CLIP || k == K_BLEND; }

// ------------------------------------------------------------- box algebra
// Intersection (clip, Sec. 6.1) and union (blend, Sec. 6.2) of (x0,y0,x1,y1)
// boxes.  min/max are exact, so any association gives the same bits.
__host__ __device__ __forceinline__ float4 box_universe() {
  return make_float4(-INFINITY, -INFINITY, INFINITY, INFINITY);
}
__host__ __device__ __forceinline__ float4 box_empty() {
  return make_float4(INFINITY, INFINITY, -INFINITY, -INFINITY);
}
__host__ __device__ __forceinline__ float4 box_isect(float4 a, float4 b) {
  return make_float4(fmaxf(a.x, b.x), fmaxf(a.y, b.y), fminf(a.z, b.z), fminf(a.w, b.w));
}
__host__ __device__ __forceinline__ float4 box_unite(float4 a, float4 b) {
  return make_float4(fminf(a.x, b.x), fminf(a.y, b.y), fmaxf(a.z, b.z), fmaxf(a.w, b.w));
}
// Empty when x0 >= x1 or y0 >= y1; empty boxes become the union identity.
__host__ __device__ __forceinline__ float4 box_canon(float4 b) {
  return (b.x >= b.z || b.y >= b.w) ? box_empty() : b;
}

struct OpAdd { __device__ int operator()(int a, int b) const { return a + b; } };
// (depth change, lowest depth reached relative to the start) of consecutive
// spans: the earlier span on the left.
struct OpDepth {
  __device__ int2 operator()(int2 a, int2 b) const {
    const int lo = a.x + b.y;
    return make_int2(a.x + b.x, a.y < lo ? a.y : lo);
  }
};
constexpr int DEPTH_NONE = 1 << 30;  // "no lowest depth yet" (identity of OpDepth)
struct OpMin { __device__ int operator()(int a, int b) const { return a < b ? a : b; } };
struct OpIsect { __device__ float4 operator()(float4 a, float4 b) const { return box_isect(a, b); } };
struct OpUnite { __device__ float4 operator()(float4 a, float4 b) const { return box_unite(a, b); } };

__device__ __forceinline__ int2 shfl_up(int2 v, int d) { return make_int2(shfl_up(v.x, d), shfl_up(v.y, d)); }

// Shuffles of any other trivially copyable value (a monoid value of the
// caller's own), 32 bits at a time.  The overloads for the built-in types
// take precedence.
template <class T, class F>
__device__ __forceinline__ T shfl_words(const T& v, F f) {
  static_assert(sizeof(T) % 4 == 0, "shuffled values are whole 32-bit words");
  unsigned w[sizeof(T) / 4];
  memcpy(w, &v, sizeof(T));
#pragma unroll
  for (int i = 0; i < (int)(sizeof(T) / 4); ++i) w[i] = f(w[i]);
  T r;
  memcpy(&r, w, sizeof(T));
  return r;
}
template <class T>
__device__ __forceinline__ T shfl_up(const T& v, int d) {
  return shfl_words(v, [d](unsigned x) { return (unsigned)shfl_up((int)x, d); });
}
template <class T>
__device__ __forceinline__ T shfl_down(const T& v, int d) {
  return shfl_words(v, [d](unsigned x) { return (unsigned)shfl_down((int)x, d); });
}
template <class T>
__device__ __forceinline__ T shfl_xor(const T& v, int m) {
  return shfl_words(v, [m](unsigned x) { return (unsigned)shfl_xor((int)x, m); });
}
template <class T>
__device__ __forceinline__ T shfl_idx(const T& v, int src) {
  return shfl_words(v, [src](unsigned x) { return (unsigned)shfl_idx((int)x, src); });
}
__device__ __forceinline__ float4 shfl_xor(float4 v, int m) {
  return make_float4(shfl_xor(v.x, m), shfl_xor(v.y, m), shfl_xor(v.z, m), shfl_xor(v.w, m));
}
__device__ __forceinline__ float4 shfl_up(float4 v, int d) {
  return make_float4(shfl_up(v.x, d), shfl_up(v.y, d), shfl_up(v.z, d), shfl_up(v.w, d));
}
__device__ __forceinline__ float4 shfl_down(float4 v, int d) {
  return make_float4(shfl_down(v.x, d), shfl_down(v.y, d), shfl_down(v.z, d), shfl_down(v.w, d));
}

// ------------------------------------------------------------ block scans
// Inclusive warp scan in lane order: lane i gets v_0 * ... * v_i (earlier
// operand on the left, so non-commutative operators are fine).
template <class T, class Op>
__device__ __forceinline__ T warp_incl_scan(T v, Op op) {
  const int lane = lane_id();
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T y = shfl_up(v, d);
    if (lane >= d) v = op(y, v);
  }
  return v;
}

// Exclusive scan over the threads of the block (NWARPS warps, NW by
// default) in thread order.  s holds NWARPS + 1 values of scratch; *total
// receives the fold of all inputs.
template <int NWARPS = NW, class T, class Op>
__device__ T block_excl_scan(T v, T ident, Op op, T* s, T* total) {
  const int lane = lane_id(), w = warp_id();
  T incl = warp_incl_scan(v, op);
  if (lane == 31) s[w] = incl;
  __syncthreads();
  if (threadIdx.x < 32) {
    T wv = threadIdx.x < NWARPS ? s[threadIdx.x] : ident;
    T wi = warp_incl_scan(wv, op);
    T we = shfl_up(wi, 1);
    if (lane == 0) we = ident;
    if (threadIdx.x < NWARPS) s[threadIdx.x] = we;
    if (threadIdx.x == 31) s[NWARPS] = wi;
  }
  __syncthreads();
  T ex = shfl_up(incl, 1);
  if (lane == 0) ex = ident;
  T r = op(s[w], ex);
  *total = s[NWARPS];
  __syncthreads();
  return r;
}

// Exclusive suffix minimum: thread j gets min over the later threads of the
// block (INT_MAX for the last thread).
template <int NWARPS = NW>
__device__ __forceinline__ int block_excl_suffix_min(int v, int* s) {
  const int lane = lane_id(), w = warp_id();
  int incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int y = shfl_down(incl, d);
    if (lane + d < 32) incl = incl < y ? incl : y;
  }
  if (lane == 0) s[w] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = INT_MAX;
    for (int i = NWARPS - 1; i >= 0; --i) {
      int x = s[i];
      s[i] = acc;
      acc = acc < x ? acc : x;
    }
  }
  __syncthreads();
  int ex = shfl_down(incl, 1);
  if (lane == 31) ex = INT_MAX;
  int after = s[w];
  int r = ex < after ? ex : after;
  __syncthreads();
  return r;
}

// Exclusive suffix fold over the NT threads in thread order: thread j gets
// v_{j+1} * ... * v_{NT-1} (ident for the last thread).  s holds NW values.
template <class T, class Op>
__device__ T block_excl_suffix(T v, T ident, Op op, T* s) {
  const int lane = lane_id(), w = warp_id();
  T incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T y = shfl_down(incl, d);
    if (lane + d < 32) incl = op(incl, y);
  }
  if (lane == 0) s[w] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    T acc = ident;
    for (int i = NW - 1; i >= 0; --i) {
      const T x = s[i];
      s[i] = acc;
      acc = op(x, acc);
    }
  }
  __syncthreads();
  T ex = shfl_down(incl, 1);
  if (lane == 31) ex = ident;
  const T r = op(ex, s[w]);
  __syncthreads();
  return r;
}

// ----------------------------------------------------------- segment trees
// Implicit tree over P leaves (P a power of two): leaves at [P, 2P), node i
// covers its children 2i and 2i+1, the root is node 1.
//
// tree_last_le: the largest leaf index u < x whose value is <= thr, or -1.
// This is the up-then-down search of the paper's core matching algorithm
// (Sec. 5, Fig. "core") run over a tree of minima instead of Bic values:
// climb while the subtree just left of the current boundary cannot contain
// an answer, then descend into the first one that can, preferring right.
template <class T>
__device__ __forceinline__ int tree_last_le(const T* tree, int P, int x, T thr) {
  if (x <= 0) return -1;
  int node;
  if (x >= P) {
    if (!(tree[1] <= thr)) return -1;
    node = 1;
  } else {
    int l = P, r = P + x;
    node = -1;
    while (l < r) {
      if (r & 1) {
        --r;
        if (tree[r] <= thr) { node = r; break; }
      }
      l >>= 1;
      r >>= 1;
    }
    if (node < 0) return -1;
  }
  while (node < P) node = (tree[2 * node + 1] <= thr) ? 2 * node + 1 : 2 * node;
  return node - P;
}

// Fold of leaves l..r (inclusive) in leaf order; ident when l > r.
template <class T, class Op>
__device__ __forceinline__ T tree_range(const T* tree, int P, int l, int r, T ident, Op op) {
  if (l > r) return ident;
  T left = ident, right = ident;
  for (l += P, r += P + 1; l < r; l >>= 1, r >>= 1) {
    if (l & 1) left = op(left, tree[l++]);
    if (r & 1) right = op(tree[--r], right);
  }
  return op(left, right);
}

// ------------------------------------------------------------- workspace
// Device view of the scratch of one scene pass.  Per tile t:
//   t_a, t_b     Bic(tile) = (unmatched closes, unmatched opens)
//   t_tot        depth change over the tile (t_b - t_a)
//   t_dstart     global depth before the tile's first element
//   t_lo         t_dstart - t_a, the lowest depth the tile reaches
//   t_ps         last earlier tile whose lo is below t_lo (owner of depth
//                t_lo - 1 in the stack at the tile start), -1 if none
//   t_q          owner of depth t_dstart - 1 (last earlier tile with
//                lo <= t_dstart - 1), -1 if none
//   t_B          clip in force at depth t_lo - 1 at the tile start
//   t_uall       union of all canonical leaf boxes of the tile
// Per tile and slot s < t_b (slot s = depth t_lo + s), at t_boff[t] + s in
// the open-side arrays (a tile's range is taken from a counter when its
// summary is written; slot_cap entries in all, enough for any balanced
// stream):
//   slice_pos    global index of the tile's unmatched open at that depth
//                (the tile's stack slice, Sec. 7.1)
//   slice_rel    intersection of the clip boxes of the slice up to slot s
//   usuf         union of the tile's leaves after that open
// A slice entry is named by its "source" u * TILE + s (owner tile u, slot
// s); slice_at() turns that into the array index.
// Per tile and m < t_a (the close that pops depth t_dstart - 1 - m), at
// t_aoff[t] + m in the close-side arrays (t_aoff = exclusive scan of t_a):
//   upre         union of the tile's leaves before that close
//   cpos         global index of that close
// ctx_src rows (tiles whose owner segments overflow) hold t_a + 1 sources
// from t_aoff[t] + t.
struct SceneWs {
  unsigned* counter;  // [1]: tile ticket of the persistent main pass; [2]: slice slots taken
  int* t_a;
  int* t_b;
  int* t_tot;         // per tile: depth change over the tile
  int* t_dstart;
  int* t_lo;
  int* t_ps;
  int* t_q;
  int* lo_tree;      // 2P
  const int* status; // status word of the call: the passes after the tile
                     // summaries stop at once when it already holds an error
  int* t_link[2];
  float4* t_val[2];
  float4* t_B;
  float4* t_uall;
  float4* uall_tree;  // union table levels 1 .. (levels - 1), T entries each
  int* slice_pos;
  float4* slice_rel;
  float4* usuf;
  float4* upre;
  int* cpos;
  int* cval;         // per tile and m: value match[open] receives (scene-local close)
  int4* t_seg;       // per tile SEGK owner segments of the stack at its start
  int* t_segb;       // per tile and segment: t_boff[owner] - owner's lowest depth (array
                     // index of the slice entry at global depth d = d + this)
  int* t_nseg;       // segment count, or SEGK + 1 when the chain continues
  int2* t_cont;      // continuation (owner, depth) when t_nseg = SEGK + 1
  int* ctx_src;      // per tile (t_a + 1): context sources, for tiles whose chain overflows
  int* t_boff;       // per tile: first open-side slot of its slice (-1: none taken)
  int* t_aoff;       // per tile: first close-side slot
  long long slot_cap;  // open-side and close-side slots available
  int T;
  int P;
};

// Array index of slice entry `src` (owner tile * TILE + slot); debug builds
// check it (and read entry 0 instead of an index outside the arrays).
__device__ __forceinline__ long long slice_at(const SceneWs& ws, int src) {
  const long long i = (long long)ws.t_boff[src / TILE] + (src % TILE);
  return in_range(i, 0, ws.slot_cap, ws.status) ? i : 0;
}

// Owner segments precomputed per tile by the tile-level resolve: segment j
// of tile t is {owner tile u (-1 below the root), u's lowest depth, lowest
// and highest global depth covered}; together they cover depths
// t_dstart - 1 - t_a .. t_dstart - 1 of the stack at the tile start.
constexpr int SEGK = 8;

// Owner segments of the stack at a tile start.  Collected by one thread, a
// bounded number at a time: segment i covers global depths
// [seg_lo[i], seg_hi[i]] owned by tile seg_u[i] (whose slice starts at depth
// seg_ulo[i]); seg_u = -1 means below the root.
constexpr int SEG_CAP = 32;
struct SegState {
  int u, dtop, dbot, n, done;
  int seg_u[SEG_CAP], seg_ulo[SEG_CAP], seg_lo[SEG_CAP], seg_hi[SEG_CAP];
};

// Starting from the owner S.u of depth S.dtop, follow the ps links (each
// tile's ps is the owner of the depth just below its own slice) down to
// depth S.dbot, recording at most SEG_CAP segments.  Every segment lowers
// S.dtop by at least one, so the batches a caller collects until S.done end;
// a segment that would not (only a workspace inconsistent with itself can
// produce one) ends the walk at once and records ST_BOUNDS in debug builds.
__device__ __forceinline__ void seg_collect(SegState& S, const int* t_ps, const int* t_lo,
                                            const int* status) {
  int n = 0;
  while (n < SEG_CAP && S.dtop >= S.dbot) {
    if (S.dtop < 0 || S.u < 0) {
      S.seg_u[n] = -1;
      S.seg_ulo[n] = 0;
      S.seg_lo[n] = S.dbot;
      S.seg_hi[n] = S.dtop;
      ++n;
      S.dtop = S.dbot - 1;
      break;
    }
    int lo_u = t_lo[S.u];
    int lo_s = lo_u > S.dbot ? lo_u : S.dbot;
    if (lo_s > S.dtop) {
      if (TB_DEBUG) atomic_cas_i32(const_cast<int*>(status), ST_OK, ST_BOUNDS);
      S.dtop = S.dbot - 1;
      break;
    }
    S.seg_u[n] = S.u;
    S.seg_ulo[n] = lo_u;
    S.seg_lo[n] = lo_s;
    S.seg_hi[n] = S.dtop;
    ++n;
    S.dtop = lo_s - 1;
    S.u = t_ps[S.u];
  }
  S.n = n;
  S.done = S.dtop < S.dbot;
}

// Segment of the current batch holding global depth d (segments are in
// decreasing depth order); -1 if outside the batch.
__device__ __forceinline__ int segk_find(const int4* seg, int n, int d) {
  for (int i = 0; i < n; ++i)
    if (d >= seg[i].z && d <= seg[i].w) return i;
  return -1;
}

__device__ __forceinline__ int seg_find(const SegState& S, int d) {
  for (int i = 0; i < S.n; ++i)
    if (d >= S.seg_lo[i] && d <= S.seg_hi[i]) return i;
  return -1;
}

}  // namespace tb

#endif  // TB_CORE_CUH
