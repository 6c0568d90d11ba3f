// tb_tree_kernels.cuh -- folds of a monoid over the tree (Sec. 1 and Sec. 13:
// the method works for any associative operation with an identity) and the
// adjoint of the 3x4 affine root-path product.
//
// Values live on the opens ("joints"), joint r being the r-th open of the
// stream (pre-order).  The joint tree is described by
//   jdepth[r]   depth of joint r (1 at a root)
//   jparent[r]  parent joint (-1 at a root): the last joint before r that is
//               shallower than r, since everything between a parent and its
//               child lies in the parent's subtree
//   jend[r]     one past the last joint of r's subtree: the first joint after
//               r that is not deeper than r (J if none), so the subtree of r
//               is the contiguous range [r, jend[r]) (Sec. 6.2)
// Both are nearest-smaller-value searches over jdepth, done with the up/down
// search of a min tree (Sec. 5, Fig. "core"): inside a tile of joints over a
// tree in shared memory, across tiles over a tree of tile minima and the
// tile's monotone prefix / suffix minima.
//
//   k_tdepth     one pass over the kinds with a decoupled look-back over the
//                element tiles' open and close counts: depth of every joint,
//                balance and kind checks
//   k_jminmax    per joint tile: prefix and suffix minima of jdepth, tile min
//   k_jmin_tree  min tree over the tiles (one block)
//   k_jstruct    per joint tile: jparent and jend; for a DOWN scan also the
//                prefix folds of the tile's exported chain (below)
//
// Joints are processed in tiles of JT = 1024 consecutive joints, one block of
// JNT threads each; thread c owns the chunk of JC = 4 joints [c*JC, c*JC+JC).
//
// DOWN (root-path fold, ancestor on the left, Sec. 6.1):
//   * A joint whose subtree runs past the end of its chunk (or tile) is
//     "exported" from it.  The exported joints of a chunk or tile form one
//     parent-child chain, and every other joint's nearest ancestor outside
//     its chunk is an exported joint of an earlier chunk.
//   * k_jstruct<CHAIN>: per tile, the prefix fold of its exported chain
//     relative to the chain's base (the parent of its first link).
//   * k_down_tiles: pointer jumping over tiles (each tile links to the tile
//     of its base) gives the fold at every tile's base.
//   * k_down_tile: in-chunk walk relative to each joint's nearest outside
//     ancestor, pointer jumping over the chunks of the tile, then every joint
//     combines its outside ancestor's fold with its own relative fold.
//
// UP (subtree fold in stream order):
//   * k_up_tile: in-chunk subtree folds by walking each joint's children,
//     folds that leave the chunk completed with a segment tree over the
//     tile's chunk totals, which is published per tile.
//   * k_up_tiles: segment tree over the tiles' totals.
//   * k_up_cross: completes the folds of subtrees that leave their tile.
//
// Affine adjoint (loss = sum_r <W_r, world_r>): world by DOWN, then
// A_r = sum over the subtree of W_d (x) world_d^T by UP, and in the same
// kernels Gbar_r = A_r world_r^{-T} and dL_r = R_parent^T Gbar_r.
//   * k_adjoint_tile: per tile, the DOWN fold of k_down_tile, the adjoint
//     values in place of the world values, the UP fold of k_up_tile and the
//     finish, in one block; then k_up_tiles and k_up_cross as for UP.
#ifndef TB_TREE_KERNELS_CUH
#define TB_TREE_KERNELS_CUH

#include "tb_core.cuh"

namespace tb {

// The tree kernels keep their own shape whatever the scene kernels are
// built with: blocks of TNT threads, TKPT elements per thread in the depth
// pass, JC joints per thread in the joint passes.
constexpr int TNT = 256;
constexpr int TNW = TNT / 32;
constexpr int TKPT = 16;
constexpr int TTILE = TNT * TKPT;
constexpr int JC = 4;          // joints per thread
#ifndef TB_TREE_JNT
#define TB_TREE_JNT 256
#endif
constexpr int JNT = TB_TREE_JNT;  // threads per joint tile
constexpr int JNW = JNT / 32;
constexpr int JT = JNT * JC;    // joints per tile
constexpr int NCH = JNT;        // chunks per tile
constexpr int NO_CHAIN = -2;   // tile without exported joints
constexpr int kMaxJumpRounds = 40;
constexpr int STRUCT_MAGIC = 0x54425354;  // header word of a complete joint structure
constexpr int ST_INVALID = 1;  // TB_ERR_INVALID_ARG

__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

// ------------------------------------------------------------- monoids
// A 3x4 affine transform [R | t] acting on column vectors, stored as three
// rows (R_i0, R_i1, R_i2, t_i).
struct Aff {
  float4 r0, r1, r2;
};

__host__ __device__ __forceinline__ Aff aff_identity() {
  Aff a;
  a.r0 = make_float4(1.f, 0.f, 0.f, 0.f);
  a.r1 = make_float4(0.f, 1.f, 0.f, 0.f);
  a.r2 = make_float4(0.f, 0.f, 1.f, 0.f);
  return a;
}
__host__ __device__ __forceinline__ Aff aff_zero() {
  Aff a;
  a.r0 = a.r1 = a.r2 = make_float4(0.f, 0.f, 0.f, 0.f);
  return a;
}
// Row i of A*B where B is applied first: (A*B)x = A(Bx).
__host__ __device__ __forceinline__ float4 aff_mul_row(float4 a, const Aff& B) {
  float4 c;
  c.x = fmaf(a.x, B.r0.x, fmaf(a.y, B.r1.x, a.z * B.r2.x));
  c.y = fmaf(a.x, B.r0.y, fmaf(a.y, B.r1.y, a.z * B.r2.y));
  c.z = fmaf(a.x, B.r0.z, fmaf(a.y, B.r1.z, a.z * B.r2.z));
  c.w = fmaf(a.x, B.r0.w, fmaf(a.y, B.r1.w, fmaf(a.z, B.r2.w, a.w)));
  return c;
}
__host__ __device__ __forceinline__ Aff aff_mul(const Aff& A, const Aff& B) {
  Aff C;
  C.r0 = aff_mul_row(A.r0, B);
  C.r1 = aff_mul_row(A.r1, B);
  C.r2 = aff_mul_row(A.r2, B);
  return C;
}
__host__ __device__ __forceinline__ float4 f4_add(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__host__ __device__ __forceinline__ Aff aff_add(const Aff& a, const Aff& b) {
  Aff c;
  c.r0 = f4_add(a.r0, b.r0);
  c.r1 = f4_add(a.r1, b.r1);
  c.r2 = f4_add(a.r2, b.r2);
  return c;
}
__device__ __forceinline__ float4 shfl_idx(float4 v, int src) {
  return make_float4(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src),
                     __shfl_sync(0xffffffffu, v.z, src), __shfl_sync(0xffffffffu, v.w, src));
}
__device__ __forceinline__ Aff shfl_idx(const Aff& a, int src) {
  Aff b;
  b.r0 = shfl_idx(a.r0, src);
  b.r1 = shfl_idx(a.r1, src);
  b.r2 = shfl_idx(a.r2, src);
  return b;
}
__device__ __forceinline__ Aff shfl_up(const Aff& a, int d) {
  Aff b;
  b.r0 = shfl_up(a.r0, d);
  b.r1 = shfl_up(a.r1, d);
  b.r2 = shfl_up(a.r2, d);
  return b;
}
__device__ __forceinline__ Aff ld_aff(const void* p, int64_t i) {
  const float4* q = reinterpret_cast<const float4*>(p) + 3 * i;
  Aff a;
  a.r0 = q[0];
  a.r1 = q[1];
  a.r2 = q[2];
  return a;
}
__device__ __forceinline__ void st_aff(void* p, int64_t i, const Aff& v) {
  float4* q = reinterpret_cast<float4*>(p) + 3 * i;
  q[0] = v.r0;
  q[1] = v.r1;
  q[2] = v.r2;
}

// A monoid: value type, identity, combine (earlier operand on the left) and
// element access in global memory.
struct MonoidAddI32 {
  using V = int;
  __device__ static V identity() { return 0; }
  __device__ static V combine(V a, V b) { return (int)((unsigned)a + (unsigned)b); }
  __device__ static V load(const void* p, int64_t i) { return reinterpret_cast<const int*>(p)[i]; }
  __device__ static void store(void* p, int64_t i, V v) { reinterpret_cast<int*>(p)[i] = v; }
};
struct MonoidIsect {
  using V = float4;
  __device__ static V identity() { return box_universe(); }
  __device__ static V combine(V a, V b) { return box_isect(a, b); }
  __device__ static V load(const void* p, int64_t i) { return reinterpret_cast<const float4*>(p)[i]; }
  __device__ static void store(void* p, int64_t i, V v) { reinterpret_cast<float4*>(p)[i] = v; }
};
struct MonoidUnion {
  using V = float4;
  __device__ static V identity() { return box_empty(); }
  __device__ static V combine(V a, V b) { return box_unite(a, b); }
  __device__ static V load(const void* p, int64_t i) { return reinterpret_cast<const float4*>(p)[i]; }
  __device__ static void store(void* p, int64_t i, V v) { reinterpret_cast<float4*>(p)[i] = v; }
};
struct MonoidAffine {
  using V = Aff;
  __device__ static V identity() { return aff_identity(); }
  __device__ static V combine(const V& a, const V& b) { return aff_mul(a, b); }
  __device__ static V load(const void* p, int64_t i) { return ld_aff(p, i); }
  __device__ static void store(void* p, int64_t i, const V& v) { st_aff(p, i, v); }
};
// Entrywise sum of 3x4 matrices (the adjoint's subtree accumulation).
struct MonoidAffSum {
  using V = Aff;
  __device__ static V identity() { return aff_zero(); }
  __device__ static V combine(const V& a, const V& b) { return aff_add(a, b); }
  __device__ static V load(const void* p, int64_t i) { return ld_aff(p, i); }
  __device__ static void store(void* p, int64_t i, const V& v) { st_aff(p, i, v); }
};

// A rigid transform: rotation by the unit quaternion q = (x, y, z, w), then
// translation t (t.w unused).  Composition A*B = (qA qB, tA + qA tB qA*): B
// first, the ancestor on the left, as for the affine transforms.  Quaternions
// multiply by Hamilton's rules (i^2 = j^2 = k^2 = ijk = -1); the rotation of
// a vector uses v + 2 u x (u x v + w v), u = (x, y, z), the expansion of
// q v q* for a unit q.
struct Rig {
  float4 q, t;
};
__host__ __device__ __forceinline__ float4 quat_mul(float4 a, float4 b) {
  return make_float4(fmaf(a.w, b.x, fmaf(a.x, b.w, fmaf(a.y, b.z, -a.z * b.y))),
                     fmaf(a.w, b.y, fmaf(-a.x, b.z, fmaf(a.y, b.w, a.z * b.x))),
                     fmaf(a.w, b.z, fmaf(a.x, b.y, fmaf(-a.y, b.x, a.z * b.w))),
                     fmaf(a.w, b.w, fmaf(-a.x, b.x, fmaf(-a.y, b.y, -a.z * b.z))));
}
__host__ __device__ __forceinline__ float4 quat_rotate(float4 q, float4 v) {
  // c = u x v + w v, then v + 2 u x c
  const float cx = fmaf(q.y, v.z, fmaf(-q.z, v.y, q.w * v.x));
  const float cy = fmaf(q.z, v.x, fmaf(-q.x, v.z, q.w * v.y));
  const float cz = fmaf(q.x, v.y, fmaf(-q.y, v.x, q.w * v.z));
  return make_float4(fmaf(2.f, fmaf(q.y, cz, -q.z * cy), v.x), fmaf(2.f, fmaf(q.z, cx, -q.x * cz), v.y),
                     fmaf(2.f, fmaf(q.x, cy, -q.y * cx), v.z), 0.f);
}
struct MonoidRigid {
  using V = Rig;
  __device__ static V identity() {
    Rig r;
    r.q = make_float4(0.f, 0.f, 0.f, 1.f);
    r.t = make_float4(0.f, 0.f, 0.f, 0.f);
    return r;
  }
  __device__ static V combine(const V& a, const V& b) {
    Rig c;
    c.q = quat_mul(a.q, b.q);
    const float4 r = quat_rotate(a.q, b.t);
    c.t = make_float4(a.t.x + r.x, a.t.y + r.y, a.t.z + r.z, 0.f);
    return c;
  }
  __device__ static V load(const void* p, int64_t i) {
    const float4* f = reinterpret_cast<const float4*>(p) + 2 * i;
    Rig r;
    r.q = f[0];
    r.t = f[1];
    return r;
  }
  __device__ static void store(void* p, int64_t i, const V& v) {
    float4* f = reinterpret_cast<float4*>(p) + 2 * i;
    f[0] = v.q;
    f[1] = v.t;
  }
};

template <class M>
struct MonoidOp {
  __device__ typename M::V operator()(const typename M::V& a, const typename M::V& b) const {
    return M::combine(a, b);
  }
};

// Shared-memory slot of joint k of a tile, chosen so that the chunk-strided
// accesses of a warp (joints c0 + i of the threads' chunks) and the
// consecutive ones (joints tid + i JNT) fall on distinct banks.  Values of up
// to 32 bytes take one padding slot per chunk.  The 48-byte affine (three
// 16-byte words) takes no padding: within each aligned group of eight joints
// the slots are rotated by the group's index, so that the eight threads of a
// quarter warp, eight chunks apart in the group index, hit eight distinct
// 16-byte bank groups; the tile then fits three DOWN blocks, or three
// adjoint blocks, per SM.
template <class V>
__host__ __device__ __forceinline__ int jslot(int k) {
  if constexpr (sizeof(V) > 32) return (k & ~7) | ((k + (k >> 3)) & 7);
  else return k + k / JC;
}
template <class V>
__host__ __device__ constexpr int jslots() { return sizeof(V) > 32 ? JT : JT + JT / JC; }
static_assert(JT % 8 == 0, "the affine slots rotate within groups of eight joints");
static_assert(JT + 1 <= 32767, "tile-local subtree ends are 16-bit");

// The values of joints [R0, R0 + cnt) into their shared slots: asynchronous
// 16-byte copies when a value is whole 16-byte words (each warp copies one
// contiguous run; wait with cp_async_wait_all before the next barrier),
// else plain loads.
template <class M>
__device__ __forceinline__ void stage_tile_values(typename M::V* s_val, const void* in, int R0, int cnt) {
  using V = typename M::V;
  if constexpr (sizeof(V) % 16 == 0) {
    constexpr int WPV = (int)(sizeof(V) / 16);
    const float4* src = reinterpret_cast<const float4*>(in) + (int64_t)R0 * WPV;
    for (int f = threadIdx.x; f < cnt * WPV; f += blockDim.x) {
      const int k = f / WPV;
      cp_async16(reinterpret_cast<float4*>(s_val + jslot<V>(k)) + (f - k * WPV), src + f);
    }
    cp_async_commit();
  } else {
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) s_val[jslot<V>(k)] = M::load(in, (int64_t)R0 + k);
  }
}

// ------------------------------------------------------------- workspace
struct TreeWs {
  // element level
  unsigned long long* lb;  // look-back words of k_tdepth, one per element tile
  unsigned* counter;       // tile ticket of k_tdepth
  unsigned* xcount;        // number of entries in xlist
  int* hdr;                // {STRUCT_MAGIC, n, J} once the joint structure below
                           // is complete for that stream (0 while it is rebuilt)
  // joint level
  int* jdepth;   // depth of joint r
  int* premin;   // per joint tile: min of jdepth over the tile up to r
  int* sufmin;   // per joint tile: min of jdepth over the tile from r on
  int* jparent;  // parent joint, -1 at a root
  int* jend;     // one past the last joint of r's subtree
  int* g_tree;   // min tree over the joint tiles' minima, 2 * PJ entries
  // DOWN
  void* relT;     // fold of a tile-exported joint relative to its tile's base
  int* t_base;    // per tile: base joint of the exported chain, -1, or NO_CHAIN
  int* t_link[2];
  void* t_val[2];
  void* t_world;  // per tile: fold at the base joint
  // UP
  void* ctree;   // per tile: its chunk segment tree, 2 * NCH values (node 1 = tile total)
  void* t_tree;  // segment tree over the tiles' totals, 2 * PJ values
  int* xlist;    // joints whose subtree leaves their tile
  int n;         // elements
  int J;         // joints (opens) announced by the caller
  int TE;        // element tiles (TTILE elements each)
  int TJ;        // joint tiles (JT joints each)
  int PJ;        // next power of two >= TJ
  int withhold;  // element tile that never publishes its look-back word
                 // (self-test of the bounded wait); -1 normally
  const int* status;  // status word of the call: the kernels after the depth
                      // pass stop at once when it already holds an error
};

// ------------------------------------------------------------- joint tree
__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) v += shfl_xor(v, m);
  return v;
}

// Look-back word of k_tdepth: flag (2 bits: 1 aggregate, 2 inclusive
// prefix) | opens (31 bits) | closes (31 bits).
__device__ __forceinline__ unsigned long long oc_pack(unsigned flag, unsigned opens, unsigned closes) {
  return ((unsigned long long)flag << 62) | ((unsigned long long)(opens & 0x7fffffffu) << 31) |
         (unsigned long long)(closes & 0x7fffffffu);
}
__device__ __forceinline__ unsigned oc_flag(unsigned long long w) { return (unsigned)(w >> 62); }
__device__ __forceinline__ unsigned oc_opens(unsigned long long w) { return (unsigned)(w >> 31) & 0x7fffffffu; }
__device__ __forceinline__ unsigned oc_closes(unsigned long long w) { return (unsigned)w & 0x7fffffffu; }

// Depth of every joint, in one pass over the kinds: open and close counts
// before each element come from a block scan plus a decoupled look-back over
// the earlier tiles (warp 0 polls 32 predecessors at a time).  Also checks
// the kinds, that the depth never drops below 0, that it ends at 0, and that
// the stream has exactly J opens.
__global__ void __launch_bounds__(TNT) k_tdepth(const uint8_t* __restrict__ kind, TreeWs w,
                                               int* status) {
  __shared__ int s_scr[TNW + 1];
  __shared__ int s_t;
  __shared__ unsigned s_o, s_c;
  const int tid = threadIdx.x;
  if (tid == 0) s_t = (int)atomic_add_u32(w.counter, 1u);
  __syncthreads();
  const int t = s_t;
  const int64_t e0 = (int64_t)t * TTILE + (int64_t)tid * TKPT;
  uint8_t kk[TKPT];
  if (e0 + TKPT <= w.n) {
    const uint4 q = ld_nc_u4(kind + e0);
    const uint32_t wds[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int i = 0; i < TKPT; ++i) kk[i] = (uint8_t)(wds[i >> 2] >> (8 * (i & 3)));
  } else {
#pragma unroll
    for (int i = 0; i < TKPT; ++i) kk[i] = e0 + i < w.n ? kind[e0 + i] : (uint8_t)K_PAD;
  }
  int co = 0, cc = 0, run = 0, mn = 0;
  bool bad = false;
#pragma unroll
  for (int i = 0; i < TKPT; ++i) {
    const int k = kk[i];
    bad |= k > K_CLOSE && k != K_PAD;
    co += kind_open(k) ? 1 : 0;
    cc += k == K_CLOSE ? 1 : 0;
    run += kind_delta(k);
    mn = mn < run ? mn : run;
  }
  if (bad) atomic_cas_i32(status, ST_OK, ST_BAD_KIND);
  int tot_o, tot_c, tile_mn;
  const int ex_o = block_excl_scan<TNW>(co, 0, OpAdd(), s_scr, &tot_o);
  const int ex_c = block_excl_scan<TNW>(cc, 0, OpAdd(), s_scr, &tot_c);
  if (tid == 0 && t != w.withhold) st_release_u64(w.lb + t, oc_pack(1u, (unsigned)tot_o, (unsigned)tot_c));
  block_excl_scan<TNW>(ex_o - ex_c + mn, INT_MAX, OpMin(), s_scr, &tile_mn);
  if (warp_id() == 0) {
    const int lane = lane_id();
    unsigned long long* lb = w.lb;
    unsigned xo = 0, xc = 0;
    bool timed_out = false;
    for (int hi = t - 1; hi >= 0; hi -= 32) {
      const int j = hi - lane;
      unsigned flag = 2u;  // before tile 0: inclusive prefix 0
      unsigned vo = 0, vc = 0;
      if (j >= 0) {
        unsigned long long v = 0;
        unsigned it = 0;
        for (;;) {
          v = ld_acquire_u64(lb + j);
          if (oc_flag(v) != 0) break;
          if (++it >= SPIN_LIMIT) break;
          poll_backoff(it);
        }
        flag = oc_flag(v);
        vo = oc_opens(v);
        vc = oc_closes(v);
        if (flag == 0u) {
          timed_out = true;
          flag = 2u;
          vo = vc = 0;
        }
      }
      const unsigned incl = ballot(flag == 2u);
      if (incl != 0u && lane > lowest_set(incl)) vo = vc = 0;
      xo += (unsigned)warp_sum_i((int)vo);
      xc += (unsigned)warp_sum_i((int)vc);
      if (incl != 0u) break;
    }
    const bool any_timeout = ballot(timed_out) != 0u;
    if (lane == 0) {
      if (any_timeout) atomic_cas_i32(status, ST_OK, ST_TIMEOUT);
      if (t != w.withhold) st_release_u64(lb + t, oc_pack(2u, xo + (unsigned)tot_o, xc + (unsigned)tot_c));
      s_o = xo;
      s_c = xc;
      const long long d0 = (long long)xo - (long long)xc;
      if (d0 + tile_mn < 0) atomic_cas_i32(status, ST_OK, ST_UNBALANCED);
      if (t == w.TE - 1) {
        if (d0 + tot_o - tot_c != 0) atomic_cas_i32(status, ST_OK, ST_UNBALANCED);
        if ((long long)xo + tot_o != (long long)w.J) atomic_cas_i32(status, ST_OK, ST_INVALID);
      }
    }
  }
  __syncthreads();
  int o = (int)s_o + ex_o, c = (int)s_c + ex_c;
#pragma unroll
  for (int i = 0; i < TKPT; ++i) {
    const int k = kk[i];
    if (kind_open(k)) {
      if (o < w.J) w.jdepth[o] = o - c + 1;
      ++o;
    } else if (k == K_CLOSE) {
      ++c;
    }
  }
}

// Per joint tile: inclusive prefix and suffix minima of jdepth, tile minimum.
__global__ void __launch_bounds__(JNT) k_jminmax(TreeWs w) {
  __shared__ int s_scr[JNW + 1];
  if (*w.status != ST_OK) return;  // the joint depths are not valid
  const int t = blockIdx.x, tid = threadIdx.x;
  const int R0 = t * JT, cnt = min(JT, w.J - R0);
  int d[JC];
  int mn = INT_MAX;
#pragma unroll
  for (int i = 0; i < JC; ++i) {
    const int k = tid * JC + i;
    d[i] = k < cnt ? w.jdepth[R0 + k] : INT_MAX;
    mn = mn < d[i] ? mn : d[i];
  }
  int all;
  int pre = block_excl_scan<JNW>(mn, INT_MAX, OpMin(), s_scr, &all);
  int suf = block_excl_suffix_min<JNW>(mn, s_scr);
  int sv[JC];
#pragma unroll
  for (int i = JC - 1; i >= 0; --i) {
    suf = suf < d[i] ? suf : d[i];
    sv[i] = suf;
  }
#pragma unroll
  for (int i = 0; i < JC; ++i) {
    const int k = tid * JC + i;
    pre = pre < d[i] ? pre : d[i];
    if (k < cnt) {
      w.premin[R0 + k] = pre;
      w.sufmin[R0 + k] = sv[i];
    }
  }
  if (tid == 0) w.g_tree[w.PJ + t] = all;
}

// Min tree over the joint tiles (one block); leaves past the last tile hold
// INT_MAX.
__global__ void __launch_bounds__(1024) k_jmin_tree(TreeWs w) {
  if (*w.status != ST_OK) return;
  const int P = w.PJ;
  for (int t = w.TJ + threadIdx.x; t < P; t += blockDim.x) w.g_tree[P + t] = INT_MAX;
  for (int h = P / 2; h >= 1; h >>= 1) {
    __syncthreads();
    for (int i = h + threadIdx.x; i < 2 * h; i += blockDim.x) {
      const int a = w.g_tree[2 * i], b = w.g_tree[2 * i + 1];
      w.g_tree[i] = a < b ? a : b;
    }
  }
}

// Smallest leaf index u >= x whose value is <= thr, or -1: the mirror of
// tree_last_le (climb to the first subtree right of the boundary that can
// hold an answer, then descend into it preferring left).
__device__ __forceinline__ int tree_first_le(const int* tree, int P, int x, int thr) {
  if (x >= P) return -1;
  int node = P + x;
  for (;;) {
    if (tree[node] <= thr) break;
    while (node & 1) {
      node >>= 1;
      if (node == 0) return -1;
    }
    ++node;
  }
  while (node < P) node = (tree[2 * node] <= thr) ? 2 * node : 2 * node + 1;
  return node - P;
}

// The exported joints of joint tile t (bits xm of each thread's chunk) form
// one chain: list them in order in shared memory, then one warp folds their
// input values 32 links at a time into relT; the chain's base (the parent of
// its first link, first_par in the thread that holds it) goes to t_base.
template <class M>
__device__ __forceinline__ void export_chain(const TreeWs& w, const void* in, int t, unsigned xm,
                                             int first_par, int* s_list, int* s_scri) {
  using V = typename M::V;
  const int tid = threadIdx.x, R0 = t * JT;
  int nx_all;
  const int off = block_excl_scan<JNW>(popc(xm), 0, OpAdd(), s_scri, &nx_all);
  {
    int o = off;
#pragma unroll
    for (int i = 0; i < JC; ++i)
      if (xm & (1u << i)) s_list[o++] = tid * JC + i;
  }
  if (xm != 0u && off == 0) w.t_base[t] = first_par;
  if (nx_all == 0 && tid == 0) w.t_base[t] = NO_CHAIN;
  __syncthreads();
  if (warp_id() == 0) {
    const int lane = lane_id();
    V carry = M::identity();
    for (int b = 0; b < nx_all; b += 32) {
      const int idx = b + lane;
      V v = idx < nx_all ? M::load(in, R0 + s_list[idx]) : M::identity();
      v = M::combine(carry, warp_incl_scan(v, MonoidOp<M>()));
      if (idx < nx_all) M::store(w.relT, R0 + s_list[idx], v);
      carry = shfl_idx(v, 31);
    }
  }
}

// Parent and subtree end of every joint of the tile; with CHAIN, also the
// prefix folds of the tile's exported chain (the input of the DOWN scan).
template <class M, bool CHAIN>
// (seven blocks of 256 threads per SM: a 2^20-joint skeleton's 1024 tiles in
// one wave)
__global__ void __launch_bounds__(JNT, 7) k_jstruct(TreeWs w, const void* __restrict__ in) {
  using V = typename M::V;
  __shared__ int s_tree[2 * JT];
  __shared__ int s_rep[JT];
  __shared__ int s_q[2 * JT];
  __shared__ int s_nq;
  __shared__ int s_scri[JNW + 1];
  if (*w.status != ST_OK) return;
  const int t = blockIdx.x, tid = threadIdx.x;
  const int R0 = t * JT, R1 = R0 + JT;
  const int cnt = min(JT, w.J - R0);
  const int* gt = w.g_tree;  // the tiles' min tree
  for (int k = tid; k < JT; k += JNT) s_tree[JT + k] = k < cnt ? w.jdepth[R0 + k] : INT_MAX;
  if (tid == 0) s_nq = 0;
  __syncthreads();
  for (int h = JT / 2; h >= 1; h >>= 1) {
    for (int i = h + tid; i < 2 * h; i += JNT) {
      const int a = s_tree[2 * i], b = s_tree[2 * i + 1];
      s_tree[i] = a < b ? a : b;
    }
    __syncthreads();
  }
  // In the tile: parent = the last earlier joint that is shallower, end = the
  // first later joint that is not deeper.  Inside the thread's chunk of JC
  // joints by direct comparison.  The joints a chunk cannot resolve are its
  // records (no shallower joint before them in the chunk: their parents are
  // the levels m_c - 1 .. df_c - 1 of the stack at the chunk start) and its
  // chain (no later joint as shallow in the chunk: levels m_c .. dl_c, one
  // joint each).  The stack levels a chunk needs are held by a few earlier
  // chunks, each covering a run of levels with its own chain; one search of
  // the tree's level of chunk minima (node NCH + c covers chunk c) per run
  // finds the next owner (the same for the chunks that pop the chain).  What
  // no chunk of the tile holds becomes one question per stack level.
  int par[JC], end[JC], dep[JC];
  const int c0 = tid * JC;
#pragma unroll
  for (int i = 0; i < JC; ++i) {
    par[i] = end[i] = -1;
    dep[i] = c0 + i < cnt ? s_tree[JT + c0 + i] : INT_MAX;
  }
  unsigned recm = 0, chm = 0;  // records, chain
#pragma unroll
  for (int i = 0; i < JC; ++i) {
#pragma unroll
    for (int j = i - 1; j >= 0; --j)
      if (par[i] < 0 && dep[j] < dep[i]) par[i] = R0 + c0 + j;
#pragma unroll
    for (int j = i + 1; j < JC; ++j)
      if (end[i] < 0 && dep[j] <= dep[i]) end[i] = R0 + c0 + j;
    if (c0 + i < cnt) {
      if (par[i] < 0) recm |= 1u << i;
      if (end[i] < 0) chm |= 1u << i;
    }
  }
  const int mc = s_tree[NCH + tid];  // chunk minimum (INT_MAX past the last joint)
  int* s_cpos = s_rep;               // chunk chains: the joint at level mc + j of chunk c
#pragma unroll
  for (int i = 0; i < JC; ++i)
    if ((chm >> i) & 1u) s_cpos[c0 + (dep[i] - mc)] = c0 + i;
  const int mt = s_tree[1];                    // tile minimum
  const int dlt = s_tree[JT + cnt - 1];        // depth of the tile's last joint
  // ends beyond the tile: one question per level of the tile's chain (mt ..
  // dlt, one joint each), slots 0 .. ne-1; parents before the tile: one slot
  // per record asking (at most one per joint), after them
  const int ne = cnt > 0 ? dlt - mt + 1 : 0;
  if (tid == 0) s_nq = ne;
  __syncthreads();  // chains written
  // parents of the records, run by run of stack levels downwards
  if (recm) {
    int cur = dep[0] - 1, pos = tid;  // the chunk's first joint is always a record
    const int need = mc - 1 > 1 ? mc - 1 : 1;
    while (cur >= need) {
      const int cc = tree_last_le(s_tree, NCH, pos, cur);
      if (cc < 0) break;
      const int mcc = s_tree[NCH + cc];
#pragma unroll
      for (int i = 0; i < JC; ++i) {
        const int l = dep[i] - 1;
        if (((recm >> i) & 1u) && l >= mcc && l <= cur) par[i] = R0 + s_cpos[cc * JC + (l - mcc)];
      }
      cur = mcc - 1;
      pos = cc;
    }
#pragma unroll
    for (int i = 0; i < JC; ++i) {
      const int l = dep[i] - 1;
      if (((recm >> i) & 1u) && l >= 1 && l <= cur) {  // the level l entry before the tile
        const int slot = atomicAdd(&s_nq, 1);
        s_q[slot] = l;
        par[i] = -2 - slot;
      }
    }
  }
  // ends of the chain, run by run of levels downwards (the chunks that pop it)
  if (chm) {
    int cur = -1, pos = tid + 1;
#pragma unroll
    for (int i = 0; i < JC; ++i)
      if ((chm >> i) & 1u) cur = dep[i];  // the last chain joint is the deepest
    while (cur >= mc) {
      const int cc = tree_first_le(s_tree, NCH, pos, cur);
      if (cc < 0) break;
      const int mcc = s_tree[NCH + cc];
#pragma unroll
      for (int i = 0; i < JC; ++i) {
        if (!((chm >> i) & 1u) || dep[i] < mcc || dep[i] > cur) continue;
        int e = -1;
#pragma unroll
        for (int q = 0; q < JC; ++q)
          if (e < 0 && s_tree[JT + cc * JC + q] <= dep[i]) e = cc * JC + q;
        end[i] = R0 + e;
      }
      cur = mcc - 1;
      pos = cc + 1;
    }
#pragma unroll
    for (int i = 0; i < JC; ++i)
      if (((chm >> i) & 1u) && dep[i] <= cur) end[i] = -2 - (dep[i] - mt);  // question of its level
  }
  for (int qi = tid; qi < ne; qi += JNT) s_q[qi] = (mt + qi) | (1 << 30);
  __syncthreads();
  // One question per thread, all in parallel: find the tile (the neighbour
  // first), then the position in that tile's monotone prefix minima (first
  // position <= thr) or suffix minima (last position <= thr) by an 8-way
  // search (eight independent probes per round).
  for (int qi = tid; qi < s_nq; qi += JNT) {
    const int qv = s_q[qi];
    const bool is_end = ((qv >> 30) & 1) != 0;
    const int thr = qv & ((1 << 30) - 1);
    int tt;
    if (is_end) {
      if (t + 1 < w.TJ && gt[w.PJ + t + 1] <= thr) tt = t + 1;
      else tt = tree_first_le(gt, w.PJ, t + 1, thr);
    } else {
      if (t > 0 && gt[w.PJ + t - 1] <= thr) tt = t - 1;
      else tt = tree_last_le(gt, w.PJ, t, thr);
    }
    int res = is_end ? w.J : -1;
    if (tt >= 0) {
      const int len = min(JT, w.J - tt * JT);
      const int* arr = (is_end ? w.premin : w.sufmin) + (size_t)tt * JT;
      // first position where the predicate turns true ("<= thr" over the
      // prefix minima, "> thr" over the suffix minima); len if it never
      // does.  Positions below lo are false, positions from hi on true.
      int lo = 0, hi = len;
      while (lo < hi) {
        const int step = (hi - lo + 7) >> 3;
        int v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int pos = lo + j * step;
          v[j] = pos < hi ? arr[pos] : 0;
        }
        int nlo = lo, nhi = hi;
        bool found = false;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int pos = lo + j * step;
          if (!found && pos < hi) {
            if (is_end ? v[j] <= thr : v[j] > thr) {
              nhi = pos;
              found = true;
            } else {
              nlo = pos + 1;
            }
          }
        }
        lo = nlo;
        hi = nhi;
      }
      // the end is that position; the parent is the position before it
      res = tt * JT + (is_end ? lo : lo - 1);
    }
    s_q[qi] = res;
  }
  __syncthreads();
  unsigned xm = 0;
#pragma unroll
  for (int i = 0; i < JC; ++i) {
    const int k = tid * JC + i;
    if (k >= cnt) continue;
    if (par[i] < -1) par[i] = s_q[-2 - par[i]];
    if (end[i] < -1) end[i] = s_q[-2 - end[i]];
    w.jparent[R0 + k] = par[i];
    w.jend[R0 + k] = end[i];
    if (end[i] > R1) xm |= 1u << i;
  }
  if (CHAIN) {
    int first_par = -1;  // parent of the tile's first exported joint
#pragma unroll
    for (int i = 0; i < JC; ++i)
      if (i == lowest_set(xm)) first_par = par[i];
    export_chain<M>(w, in, t, xm, first_par, s_q, s_scri);
  }
}

// DOWN input of one joint tile from its joint structure alone (jparent and
// jend already in the workspace, checked against the header): the prefix
// folds of the tile's exported chain, as k_jstruct<M, true> computes them.
template <class M>
__global__ void __launch_bounds__(JNT) k_jchain(TreeWs w, const void* __restrict__ in, int* status) {
  __shared__ int s_list[JT];
  __shared__ int s_scri[JNW + 1];
  if (*w.status != ST_OK) return;
  if (w.hdr[0] != STRUCT_MAGIC || w.hdr[1] != w.n || w.hdr[2] != w.J) {
    if (threadIdx.x == 0) atomic_cas_i32(status, ST_OK, ST_INVALID);
    return;  // no complete structure for this stream in the workspace
  }
  const int t = blockIdx.x, tid = threadIdx.x;
  const int R0 = t * JT, R1 = R0 + JT;
  const int cnt = min(JT, w.J - R0);
  unsigned xm = 0;
  int first_par = -1;
#pragma unroll
  for (int i = 0; i < JC; ++i) {
    const int k = tid * JC + i;
    if (k < cnt && w.jend[R0 + k] > R1) {
      if (xm == 0u) first_par = w.jparent[R0 + k];
      xm |= 1u << i;
    }
  }
  export_chain<M>(w, in, t, xm, first_par, s_list, s_scri);
}

// Left sibling of every joint (the previous joint with the same parent, -1
// for a first child; the caller fills `left` with -1 first): the subtree of
// joint q ends at jend[q], the first later joint not deeper than q; when that
// joint is exactly as deep, everything between is inside q, so the two share
// q's parent and q is its left sibling.  Each joint has at most one such q.
__global__ void k_left_sibling(TreeWs w, int* __restrict__ left) {
  if (*w.status != ST_OK) return;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < w.J; q += gridDim.x * blockDim.x) {
    const int e = w.jend[q];
    if (e < w.J && in_range(e, q + 1, w.J, w.status) && w.jdepth[e] == w.jdepth[q]) left[e] = q;
  }
}

// ------------------------------------------------------------- DOWN
// Pointer jumping over the tiles (one block): the fold at each tile's base is
// the fold at its base's tile base times the base's chain prefix.  With SM
// the link and value buffers live in shared memory (down_tiles_smem bytes),
// otherwise in the workspace.
template <class M>
constexpr size_t down_tiles_smem(int TJ) {
  return (size_t)2 * TJ * (sizeof(typename M::V) + sizeof(int));
}

template <class M, bool SM>
__global__ void __launch_bounds__(1024) k_down_tiles(TreeWs w, int* status) {
  using V = typename M::V;
  TB_DYNAMIC_SMEM(smem);
  if (*w.status != ST_OK) return;
  if (threadIdx.x == 0) {  // the joint structure (k_jstruct) is complete
    w.hdr[1] = w.n;
    w.hdr[2] = w.J;
    w.hdr[0] = STRUCT_MAGIC;
  }
  const int TJ = w.TJ;
  V* sv = reinterpret_cast<V*>(smem);              // values of buffers 0 and 1
  int* sl = reinterpret_cast<int*>(sv + 2 * TJ);  // links of buffers 0 and 1
  auto link = [&](int buf, int t) -> int& { return SM ? sl[buf * TJ + t] : w.t_link[buf][t]; };
  auto val = [&](int buf, int t) -> V { return SM ? sv[buf * TJ + t] : M::load(w.t_val[buf], t); };
  auto set_val = [&](int buf, int t, const V& v) {
    if (SM) sv[buf * TJ + t] = v;
    else M::store(w.t_val[buf], t, v);
  };
  // world base of tile t = world base of tile link(t) times v(t), link(t) < t:
  // pointer jumping, first over the links inside each warp's run of 32 tiles
  // (shuffles, no barrier and no round trip through the link and value
  // buffers, which live in the workspace when the tiles are many), then over
  // the block
  bool bad = false;
  const int lane = threadIdx.x & 31;
  for (int tb = threadIdx.x & ~31; tb < TJ; tb += blockDim.x) {  // warp-uniform
    const int t = tb + lane;
    int l = -1;
    V v = M::identity();
    if (t < TJ) {
      const int b = w.t_base[t];
      if (b >= 0) {
        l = b / JT;
        if (l >= t) {
          l = -1;
          bad = true;
        } else {
          v = M::load(w.relT, b);
        }
      }
    }
    for (int round = 0; round < 5 && ballot(l >= tb) != 0u; ++round) {
      const int src = l >= tb ? l - tb : lane;
      const V lv = shfl_idx(v, src);
      const int ll = shfl_idx(l, src);
      if (l >= tb) {
        v = M::combine(lv, v);
        l = ll;
      }
    }
    if (t < TJ) {
      link(0, t) = l;
      set_val(0, t, v);
      if (l < 0) M::store(w.t_world, t, v);
    }
  }
  if (bad) atomic_cas_i32(status, ST_OK, ST_INVALID);
  int cur = 0;
  for (int round = 0; round < kMaxJumpRounds; ++round) {
    __syncthreads();
    bool any = false;
    for (int t = threadIdx.x; t < TJ; t += blockDim.x) {
      const int l = link(cur, t);
      V v = val(cur, t);
      int nl = -1;
      if (l >= 0) {
        v = M::combine(val(cur, l), v);
        nl = link(cur, l);
        if (nl < 0) M::store(w.t_world, t, v);
        else any = true;
      }
      link(cur ^ 1, t) = nl;
      set_val(cur ^ 1, t, v);
    }
    cur ^= 1;
    if (!block_or(any)) break;
  }
}

// The JC entries of joint array a for the chunk starting at joint cs (one
// 16-byte load when the chunk is whole: cs is a multiple of JC and the
// workspace arrays start on 256-byte boundaries); -1 past joint n.
__device__ __forceinline__ void load_chunk_ints(const int* __restrict__ a, int cs, int n, int (&v)[JC]) {
  if (JC == 4 && cs + JC <= n) {
    const int4 q = *reinterpret_cast<const int4*>(a + cs);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
  } else {
#pragma unroll
    for (int i = 0; i < JC; ++i) v[i] = cs + i < n ? a[cs + i] : -1;
  }
}

template <class M>
__device__ __forceinline__ typename M::V fold_outside(const TreeWs& w, int a) {
  return M::combine(M::load(w.t_world, a / JT), M::load(w.relT, a));
}

template <class M>
constexpr size_t down_tile_smem() {
  return (size_t)jslots<typename M::V>() * sizeof(typename M::V) + (size_t)NCH * sizeof(typename M::V) +
         (size_t)NCH * sizeof(int);
}

// The DOWN fold of joint tile R0 / JT (cnt joints): the world value of every
// joint in its shared slot when it returns (after a barrier).  s_cm and s_cl
// hold NCH values and NCH ints of scratch; par and e return the parents and
// subtree ends of the thread's chunk.
template <class M>
__device__ __forceinline__ void down_tile_fold(const TreeWs& w, const void* __restrict__ in,
                                               typename M::V* s_val, typename M::V* s_cm, int* s_cl,
                                               int R0, int cnt, int (&par)[JC], int (&e)[JC]) {
  using V = typename M::V;
  const int tid = threadIdx.x;
  stage_tile_values<M>(s_val, in, R0, cnt);
  // While the tile's values arrive: the chunk's parents and subtree ends,
  // each joint's nearest ancestor outside the chunk (from the parents alone),
  // and the world values in earlier tiles below which the chunk hangs.
  const int c0 = tid * JC;
  const int cs = R0 + c0, cend = cs + JC;  // global range of the chunk
  int anc[JC];
  unsigned xm = 0, inm = 0;  // exported joints; parent inside the chunk
  {
    load_chunk_ints(w.jparent, cs, w.J, par);
    load_chunk_ints(w.jend, cs, w.J, e);
#pragma unroll
    for (int i = 0; i < JC; ++i) {
      anc[i] = par[i];
      if (par[i] >= cs && in_range(par[i], cs, cs + i, w.status)) {  // parent before i in the chunk
        inm |= 1u << i;
#pragma unroll
        for (int j = 0; j < i; ++j)
          if (par[i] == cs + j) anc[i] = anc[j];
      }
      if (c0 + i < cnt && e[i] > cend) xm |= 1u << i;
    }
  }
  // The exported joints of a chunk hang below one base joint, the nearest
  // outside ancestor of the first of them.  A base in an earlier tile is
  // final: its world value is that tile's world fold times its relative
  // fold.  So is the nearest outside ancestor of the chunk's other joints
  // when it lies in an earlier tile (one such ancestor is loaded here, any
  // other where it is used).
  int abase = -1, apre = -1;
  if (xm) {
    int a = -1;
#pragma unroll
    for (int i = JC - 1; i >= 0; --i)
      if ((xm >> i) & 1u) a = anc[i];  // the first exported joint's
    if (in_range(a, -1, cs, w.status)) abase = a;
    // (debug builds: an ancestor at or after the chunk; left at the identity)
  }
#pragma unroll
  for (int i = 0; i < JC; ++i)
    if (apre < 0 && c0 + i < cnt && !(xm & (1u << i)) && anc[i] >= 0 && anc[i] < R0) apre = anc[i];
  V m = M::identity(), fpre = M::identity();
  if (abase >= 0 && abase < R0) m = fold_outside<M>(w, abase);
  if (apre >= 0) fpre = apre == abase ? m : fold_outside<M>(w, apre);
  cp_async_wait_all();
  __syncthreads();

  // In-chunk walk: fold relative to the nearest ancestor outside the chunk;
  // then the joints below a joint of an earlier tile take its world value.
#pragma unroll
  for (int i = 0; i < JC; ++i)
    if ((inm >> i) & 1u)
      s_val[jslot<V>(c0 + i)] = M::combine(s_val[jslot<V>(par[i] - R0)], s_val[jslot<V>(c0 + i)]);
#pragma unroll
  for (int i = 0; i < JC; ++i) {
    if (c0 + i < cnt && !(xm & (1u << i)) && anc[i] >= 0 && anc[i] < R0) {
      const V f = anc[i] == apre ? fpre : fold_outside<M>(w, anc[i]);
      s_val[jslot<V>(c0 + i)] = M::combine(f, s_val[jslot<V>(c0 + i)]);
    }
  }
  __syncthreads();
  int link = -1;
  if (abase >= R0) {
    link = (abase - R0) / JC;
    m = s_val[jslot<V>(abase - R0)];
  }
  // base of chunk c = base of chunk link(c) times m(c), link(c) < c: pointer
  // jumping, first over the links inside the warp (shuffles, no barrier;
  // the chain inside a warp halves every round), then over the block
  {
    const int wbase = tid & ~31, lane = tid & 31;
    for (int round = 0; round < 5 && ballot(link >= wbase) != 0u; ++round) {
      const int src = link >= wbase ? link - wbase : lane;
      const V lm = shfl_idx(m, src);
      const int ll = shfl_idx(link, src);
      if (link >= wbase) {
        m = M::combine(lm, m);
        link = ll;
      }
    }
  }
  s_cm[tid] = m;
  s_cl[tid] = link;
  for (int round = 0; round < kMaxJumpRounds; ++round) {
    if (!block_or(link >= 0)) break;
    int nl = -1;
    V nm = m;
    if (link >= 0) {
      nm = M::combine(s_cm[link], m);
      nl = s_cl[link];
    }
    __syncthreads();
    link = nl;
    m = nm;
    s_cm[tid] = m;
    s_cl[tid] = link;
  }
  // Exported joints: base fold times the relative fold.
#pragma unroll
  for (int i = 0; i < JC; ++i)
    if (xm & (1u << i)) s_val[jslot<V>(c0 + i)] = M::combine(m, s_val[jslot<V>(c0 + i)]);
  __syncthreads();
  // Every other joint whose outside ancestor is an exported joint of an
  // earlier chunk of this tile (final by now); those below a joint of an
  // earlier tile are done, the roots have no ancestor.
#pragma unroll
  for (int i = 0; i < JC; ++i) {
    const int k = c0 + i;
    if (k < cnt && !(xm & (1u << i))) {
      const int a = anc[i];
      if (a >= R0 && in_range(a, R0, cs, w.status))
        s_val[jslot<V>(k)] = M::combine(s_val[jslot<V>(a - R0)], s_val[jslot<V>(k)]);
      // (debug builds: an ancestor at or after the chunk is left as it is)
    }
  }
  __syncthreads();
}

template <class M>
__global__ void __launch_bounds__(JNT, 3) k_down_tile(TreeWs w, const void* __restrict__ in,
                                                     void* __restrict__ out) {
  using V = typename M::V;
  TB_DYNAMIC_SMEM(smem);
  V* s_val = reinterpret_cast<V*>(smem);
  V* s_cm = s_val + jslots<V>();
  int* s_cl = reinterpret_cast<int*>(s_cm + NCH);
  if (*w.status != ST_OK) return;
  const int R0 = blockIdx.x * JT;
  const int cnt = min(JT, w.J - R0);
  int par[JC], e[JC];
  down_tile_fold<M>(w, in, s_val, s_cm, s_cl, R0, cnt, par, e);
  for (int k = threadIdx.x; k < cnt; k += JNT) M::store(out, R0 + k, s_val[jslot<V>(k)]);
}

// ------------------------------------------------------------- adjoint
// Inverse of the 3x3 part (adjugate over determinant).
__device__ __forceinline__ void inv3(const Aff& a, float m[3][3]) {
  const float a00 = a.r0.x, a01 = a.r0.y, a02 = a.r0.z;
  const float a10 = a.r1.x, a11 = a.r1.y, a12 = a.r1.z;
  const float a20 = a.r2.x, a21 = a.r2.y, a22 = a.r2.z;
  const float c00 = a11 * a22 - a12 * a21, c01 = a12 * a20 - a10 * a22, c02 = a10 * a21 - a11 * a20;
  const float id = 1.0f / (a00 * c00 + a01 * c01 + a02 * c02);
  m[0][0] = c00 * id;
  m[1][0] = c01 * id;
  m[2][0] = c02 * id;
  m[0][1] = (a02 * a21 - a01 * a22) * id;
  m[1][1] = (a00 * a22 - a02 * a20) * id;
  m[2][1] = (a01 * a20 - a00 * a21) * id;
  m[0][2] = (a01 * a12 - a02 * a11) * id;
  m[1][2] = (a02 * a10 - a00 * a12) * id;
  m[2][2] = (a00 * a11 - a01 * a10) * id;
}

// Gbar_r = A_r world_r^{-T} = [(A^R - A^t t^T) R^{-T} | A^t] and
// dL_r = R_parent^T Gbar_r (Gbar_r itself at a root).
__device__ __forceinline__ Aff adjoint_grad(const Aff& A, const Aff& Wr, const Aff* Wp) {
  float inv[3][3];
  inv3(Wr, inv);
  const float tx = Wr.r0.w, ty = Wr.r1.w, tz = Wr.r2.w;
  const float4 arow[3] = {A.r0, A.r1, A.r2};
  float4 g[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float4 a = arow[i];
    const float b0 = a.x - a.w * tx, b1 = a.y - a.w * ty, b2 = a.z - a.w * tz;
    g[i].x = fmaf(b0, inv[0][0], fmaf(b1, inv[0][1], b2 * inv[0][2]));
    g[i].y = fmaf(b0, inv[1][0], fmaf(b1, inv[1][1], b2 * inv[1][2]));
    g[i].z = fmaf(b0, inv[2][0], fmaf(b1, inv[2][1], b2 * inv[2][2]));
    g[i].w = a.w;
  }
  Aff D;
  if (Wp != nullptr) {
    const Aff& P = *Wp;
    // row i of D = sum_k R_p[k][i] * row k of Gbar
    const float q[3][3] = {{P.r0.x, P.r1.x, P.r2.x}, {P.r0.y, P.r1.y, P.r2.y}, {P.r0.z, P.r1.z, P.r2.z}};
    float4 d[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      d[i].x = fmaf(q[i][0], g[0].x, fmaf(q[i][1], g[1].x, q[i][2] * g[2].x));
      d[i].y = fmaf(q[i][0], g[0].y, fmaf(q[i][1], g[1].y, q[i][2] * g[2].y));
      d[i].z = fmaf(q[i][0], g[0].z, fmaf(q[i][1], g[1].z, q[i][2] * g[2].z));
      d[i].w = fmaf(q[i][0], g[0].w, fmaf(q[i][1], g[1].w, q[i][2] * g[2].w));
    }
    D.r0 = d[0];
    D.r1 = d[1];
    D.r2 = d[2];
  } else {
    D.r0 = g[0];
    D.r1 = g[1];
    D.r2 = g[2];
  }
  return D;
}

// What the UP kernels do with a completed subtree fold besides storing it:
// nothing, or turn the adjoint's A_r into grad_local[r].
// A finish reads its inputs (load, given the joint's parent) apart from
// using them (apply), so that a caller can have several joints' reads in
// flight at once.
struct NoFinish {
  static constexpr bool active = false;
  struct In {};
  __device__ In load(const TreeWs&, int, int, int) const { return In{}; }
  template <class V>
  __device__ void apply(int, const V&, const In&) const {}
  template <class V>
  __device__ void operator()(const TreeWs&, int, const V&) const {}
};
struct AdjointFinish {
  static constexpr bool active = true;
  const void* world;
  void* grad_local;
  struct In {
    Aff Wr, Wp;
    bool root;
  };
  // (a parent before own_lo takes its world value from the tile pass's
  // folds instead: its tile's world fold times its relative fold)
  __device__ In load(const TreeWs& w, int r, int p, int own_lo) const {
    In x;
    x.Wr = ld_aff(world, r);
    x.root = p < 0;
    if (p >= own_lo) x.Wp = ld_aff(world, p);
    else if (p >= 0) x.Wp = fold_outside<MonoidAffine>(w, p);
    return x;
  }
  __device__ void apply(int r, const Aff& A, const In& x) const {
    st_aff(grad_local, r, adjoint_grad(A, x.Wr, x.root ? nullptr : &x.Wp));
  }
  __device__ void operator()(const TreeWs& w, int r, const Aff& A) const {
    apply(r, A, load(w, r, w.jparent[r], 0));
  }
};

// ------------------------------------------------------------- UP
// Fold of leaves l..r (inclusive) of a segment tree with P leaves; node(i)
// returns node i.
template <class M, class Node>
__device__ __forceinline__ typename M::V seg_fold(Node node, int P, int l, int r) {
  using V = typename M::V;
  V left = M::identity(), right = M::identity();
  if (l > r) return left;
  for (l += P, r += P + 1; l < r; l >>= 1, r >>= 1) {
    if (l & 1) left = M::combine(left, node(l++));
    if (r & 1) right = M::combine(node(--r), right);
  }
  return M::combine(left, right);
}

// Values of the UP pass: the caller's input, or the adjoint's
// X_r = W_r (x) world_r^T = [W^R R^T + W^t t^T | W^t].
template <class M>
struct InputValues {
  const void* in;
  __device__ typename M::V operator()(int r) const { return M::load(in, r); }
};
struct AdjointValues {
  const void* grad_world;
  const void* world;
  __device__ static float4 row(float4 g, const Aff& W) {
    float4 x;
    x.x = fmaf(g.x, W.r0.x, fmaf(g.y, W.r0.y, fmaf(g.z, W.r0.z, g.w * W.r0.w)));
    x.y = fmaf(g.x, W.r1.x, fmaf(g.y, W.r1.y, fmaf(g.z, W.r1.z, g.w * W.r1.w)));
    x.z = fmaf(g.x, W.r2.x, fmaf(g.y, W.r2.y, fmaf(g.z, W.r2.z, g.w * W.r2.w)));
    x.w = g.w;
    return x;
  }
  __device__ static Aff apply(const Aff& G, const Aff& W) {
    Aff X;
    X.r0 = row(G.r0, W);
    X.r1 = row(G.r1, W);
    X.r2 = row(G.r2, W);
    return X;
  }
  __device__ Aff operator()(int r) const { return apply(ld_aff(grad_world, r), ld_aff(world, r)); }
};

template <class M>
constexpr size_t up_tile_smem() {
  return (size_t)jslots<typename M::V>() * sizeof(typename M::V) + (size_t)2 * NCH * sizeof(typename M::V) +
         (size_t)JT * sizeof(short);
}

// The UP fold of joint tile R0 / JT (cnt joints) from its values in s_val
// and its tile-local subtree ends in s_end (both complete, after a barrier):
// every joint's fold over its subtree within the tile in its slot when it
// returns (after a barrier); the chunk tree (2 NCH values of scratch in
// s_tree) goes to the workspace, the joints leaving the tile to its list.
template <class M>
__device__ __forceinline__ void up_tile_fold(const TreeWs& w, typename M::V* s_val, typename M::V* s_tree,
                                             const short* s_end, int R0, int cnt) {
  using V = typename M::V;
  const int t = R0 / JT, tid = threadIdx.x;
  const int c0 = tid * JC, ce = c0 + JC;
  const int lim = min(ce, cnt);
  // Joints whose subtree leaves the tile go to the list k_up_cross serves:
  // one atomic per warp for the warp's entries (issued first: only the ends
  // are needed, and the atomic's latency then overlaps the walks below).
  {
    unsigned xm = 0;
    for (int k = c0; k < lim; ++k)
      if (s_end[k] > JT) xm |= 1u << (k - c0);
    const int nx = popc(xm);
    int incl = nx;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int o = shfl_up(incl, d);
      if (lane_id() >= d) incl += o;
    }
    const int wtot = shfl_idx(incl, 31);
    if (wtot > 0) {
      unsigned wbase = 0;
      if (lane_id() == 31) wbase = atomic_add_u32(w.xcount, (unsigned)wtot);
      wbase = (unsigned)shfl_idx((int)wbase, 31);
      unsigned at = wbase + (unsigned)(incl - nx);
      for (unsigned m = xm; m; m &= m - 1) w.xlist[at++] = R0 + c0 + lowest_set(m);
    }
  }
  // Walk the chunk backwards: a joint's fold is its own value followed by its
  // children's folds; a child leaving the chunk contributes its suffix.
  for (int k = lim - 1; k >= c0; --k) {
    V acc = s_val[jslot<V>(k)];
    const int stop = min(s_end[k], ce);
    for (int c = k + 1; c < stop; c = s_end[c]) {
      acc = M::combine(acc, s_val[jslot<V>(c)]);
      if (!in_range(s_end[c], c + 1, (long long)w.J - R0 + 1, w.status)) break;  // ends lie after the joint
    }
    s_val[jslot<V>(k)] = acc;
  }
  V tot = M::identity();
  for (int c = c0; c < lim; c = s_end[c]) {
    tot = M::combine(tot, s_val[jslot<V>(c)]);
    if (!in_range(s_end[c], c + 1, (long long)w.J - R0 + 1, w.status)) break;
  }
  s_tree[NCH + tid] = tot;
  __syncthreads();
  for (int h = NCH / 2; h >= 1; h >>= 1) {
    if (tid < h) s_tree[h + tid] = M::combine(s_tree[2 * (h + tid)], s_tree[2 * (h + tid) + 1]);
    __syncthreads();
  }
  // The chunk tree, for subtrees of earlier tiles ending here (their end
  // tile's prefix over whole chunks) and for the tile total (stored now, so
  // that the stores drain during the folds below).
  for (int i = tid; i < 2 * NCH; i += JNT)
    if (i > 0) M::store(w.ctree, (int64_t)t * 2 * NCH + i, s_tree[i]);
  // Joints whose subtree leaves the chunk: its in-chunk fold, the whole
  // chunks up to the one holding its end (all chunks after this one when the
  // subtree leaves the tile), then the joints of that chunk before the end.
  // These joints are nested, so taken innermost (last) first their end
  // chunks only grow: the fold over whole chunks is extended, not redone.
  auto node = [s_tree](int i) { return s_tree[i]; };
  {
    V R = M::identity();  // fold of chunks tid + 1 .. cr - 1
    int cr = tid + 1;
    for (int k = lim - 1; k >= c0; --k) {
      const int e = s_end[k];
      if (e <= ce) continue;
      const int c2 = e <= JT ? e / JC : NCH;
      if (c2 > cr) {
        R = M::combine(R, seg_fold<M>(node, NCH, cr, c2 - 1));
        cr = c2;
      }
      V acc = M::combine(s_val[jslot<V>(k)], R);
      if (e <= JT) {
        for (int j = c2 * JC; j < e; j = s_end[j]) {
          acc = M::combine(acc, s_val[jslot<V>(j)]);
          if (!in_range(s_end[j], j + 1, (long long)w.J - R0 + 1, w.status)) break;
        }
      }
      s_val[jslot<V>(k)] = acc;
    }
  }
  __syncthreads();  // every chunk's folds are complete before they are stored
}

// Stores the folds of the tile's joints (with a finish, only the partial
// folds of the subtrees leaving the tile are needed later; the others are
// finished here, two joints' finish reads in flight at a time).  pr holds
// the parents of the joints tid + i JNT; the finish reads the world values
// of joints from own_lo on from the workspace (see the finish).
template <class M, class Finish>
__device__ __forceinline__ void up_tile_store(const TreeWs& w, void* __restrict__ out, const Finish& fin,
                                              const typename M::V* s_val, const short* s_end,
                                              const int (&pr)[JT / JNT], int R0, int cnt, int own_lo) {
  using V = typename M::V;
  const int tid = threadIdx.x;
  constexpr int NI = JT / JNT;
  static_assert(NI % 2 == 0, "the finish loop takes joints in pairs");
#pragma unroll
  for (int i0 = 0; i0 < NI; i0 += 2) {
    typename Finish::In x[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int k = tid + (i0 + j) * JNT;
      if (Finish::active && k < cnt && s_end[k] <= JT) x[j] = fin.load(w, R0 + k, pr[i0 + j], own_lo);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int k = tid + (i0 + j) * JNT;
      if (k < cnt) {
        const V A = s_val[jslot<V>(k)];
        if (!Finish::active || s_end[k] > JT) M::store(out, R0 + k, A);
        if (Finish::active && s_end[k] <= JT) fin.apply(R0 + k, A, x[j]);
      }
    }
  }
}

template <class M, class Values, class Finish>
__global__ void __launch_bounds__(JNT, 2) k_up_tile(TreeWs w, Values values, void* __restrict__ out,
                                                   Finish fin) {
  using V = typename M::V;
  TB_DYNAMIC_SMEM(smem);
  V* s_val = reinterpret_cast<V*>(smem);
  V* s_tree = s_val + jslots<V>();  // chunk totals at [NCH, 2 NCH)
  short* s_end = reinterpret_cast<short*>(s_tree + 2 * NCH);  // local subtree ends (JT + 1: past the tile)
  if (*w.status != ST_OK) return;
  const int t = blockIdx.x, tid = threadIdx.x;
  const int R0 = t * JT;
  const int cnt = min(JT, w.J - R0);
  constexpr int NI = JT / JNT;
  int pr[NI];  // parents of the joints this thread finishes (a finish only)
#pragma unroll
  for (int i = 0; i < NI; ++i) {  // unrolled: every load of the tile in flight at once
    const int k = tid + i * JNT;
    pr[i] = -1;
    if (k < cnt) {
      s_val[jslot<V>(k)] = values(R0 + k);
      s_end[k] = (short)min(w.jend[R0 + k] - R0, JT + 1);
      if (Finish::active) pr[i] = w.jparent[R0 + k];
    }
  }
  __syncthreads();
  up_tile_fold<M>(w, s_val, s_tree, s_end, R0, cnt);
  up_tile_store<M>(w, out, fin, s_val, s_end, pr, R0, cnt, 0);
}

// The adjoint of the affine DOWN scan for one joint tile in one pass: the
// tile's world values (the DOWN fold; stored to the workspace for the
// cross-tile completion and the finish), then in place the adjoint values
// (AdjointValues), their UP fold and the finish.  A parent in an earlier
// tile takes its world value from the tile pass's folds, since that tile's
// block may still be running.  Shared memory: the tile's values, its local
// subtree ends, and the DOWN's chunk bases and links, later the UP's chunk
// tree.
constexpr size_t adjoint_tile_smem() {
  return (size_t)jslots<Aff>() * sizeof(Aff) + (size_t)JT * sizeof(short) + (size_t)2 * NCH * sizeof(Aff);
}
static_assert((size_t)NCH * sizeof(Aff) + (size_t)NCH * sizeof(int) <= (size_t)2 * NCH * sizeof(Aff),
              "the DOWN's scratch fits where the chunk tree goes");

__global__ void __launch_bounds__(JNT, 3) k_adjoint_tile(TreeWs w, const void* __restrict__ local,
                                                        const void* __restrict__ grad_world, void* world,
                                                        void* __restrict__ acc, AdjointFinish fin) {
  using V = Aff;
  TB_DYNAMIC_SMEM(smem);
  V* s_val = reinterpret_cast<V*>(smem);
  short* s_end = reinterpret_cast<short*>(s_val + jslots<V>());  // local subtree ends (JT + 1: past the tile)
  V* s_scr = reinterpret_cast<V*>(s_end + JT);
  if (*w.status != ST_OK) return;
  const int tid = threadIdx.x;
  const int R0 = blockIdx.x * JT;
  const int cnt = min(JT, w.J - R0);
  int par[JC], e[JC];
  down_tile_fold<MonoidAffine>(w, local, s_val, s_scr, reinterpret_cast<int*>(s_scr + NCH), R0, cnt, par, e);
  const int c0 = tid * JC;
#pragma unroll
  for (int i = 0; i < JC; ++i)
    if (c0 + i < cnt) s_end[c0 + i] = (short)min(e[i] - R0, JT + 1);
  constexpr int NI = JT / JNT;
  int pr[NI];
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    const int k = tid + i * JNT;
    pr[i] = -1;
    if (k < cnt) {
      const V W = s_val[jslot<V>(k)];
      st_aff(world, R0 + k, W);
      s_val[jslot<V>(k)] = AdjointValues::apply(ld_aff(grad_world, R0 + k), W);
      pr[i] = w.jparent[R0 + k];
    }
  }
  __syncthreads();
  up_tile_fold<MonoidAffSum>(w, s_val, s_scr, s_end, R0, cnt);
  up_tile_store<MonoidAffSum>(w, acc, fin, s_val, s_end, pr, R0, cnt, R0);
}

// Segment tree over the tiles' totals (one block).
template <class M>
__global__ void __launch_bounds__(1024) k_up_tiles(TreeWs w) {
  using V = typename M::V;
  if (*w.status != ST_OK) return;
  if (threadIdx.x == 0) {  // the joint structure (k_jstruct) is complete
    w.hdr[1] = w.n;
    w.hdr[2] = w.J;
    w.hdr[0] = STRUCT_MAGIC;
  }
  const int P = w.PJ;
  for (int t = threadIdx.x; t < P; t += blockDim.x)
    M::store(w.t_tree, P + t,
             t < w.TJ ? M::load(w.ctree, (int64_t)t * 2 * NCH + 1) : M::identity());
  for (int h = P / 2; h >= 1; h >>= 1) {
    __syncthreads();
    for (int i = h + threadIdx.x; i < 2 * h; i += blockDim.x) {
      const V v = M::combine(M::load(w.t_tree, 2 * i), M::load(w.t_tree, 2 * i + 1));
      M::store(w.t_tree, i, v);
    }
  }
}

// Fold of leaves l..r (inclusive) of a segment tree with P leaves, its node
// reads eight at a time: the nodes of the range are, in fold order, the left
// nodes of levels 0, 1, ... (level k: ceil((l + P) / 2^k) when odd) and then
// the right nodes from the top level down (level k: floor((r + P + 1) / 2^k)
// - 1 when that quotient is odd), over the levels where the range is still
// open; each batch's reads are independent, so their latencies overlap.
template <class M, class Node>
__device__ __forceinline__ typename M::V seg_fold_batched(Node node, int P, int l, int r) {
  using V = typename M::V;
  V acc = M::identity();
  if (l > r) return acc;
  const int L0 = l + P, R1 = r + P + 1;
  int nlev = 0;  // levels 0 .. nlev - 1 are open
  while (nlev < 31 && ((L0 + (1 << nlev) - 1) >> nlev) < (R1 >> nlev)) ++nlev;
  const int slots = 2 * nlev;
  for (int s0 = 0; s0 < slots; s0 += 8) {
    V v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int sl = s0 + j;
      const int k = sl < nlev ? sl : slots - 1 - sl;
      const int lk = (L0 + (1 << k) - 1) >> k, rk = R1 >> k;
      int nd = 0;
      if (sl < nlev) nd = (lk & 1) ? lk : 0;
      else if (sl < slots) nd = (rk & 1) ? rk - 1 : 0;
      v[j] = nd > 0 ? node(nd) : M::identity();
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) acc = M::combine(acc, v[j]);
  }
  return acc;
}

// Completes the folds of the subtrees that leave their tile: the partial fold
// written by k_up_tile, the whole tiles in between, and the prefix of the
// tile where the subtree ends (its whole chunks, then the joints of the chunk
// holding the end).  One thread per subtree; the reads that do not depend on
// one another are issued together.
template <class M, class Values, class Finish>
__global__ void __launch_bounds__(128) k_up_cross(TreeWs w, Values values, void* __restrict__ out,
                                                  Finish fin) {
  using V = typename M::V;
  if (*w.status != ST_OK) return;
  const int count = (int)*w.xcount;
  const void* tree = w.t_tree;
  auto node = [tree](int i) { return M::load(tree, i); };
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const int r = w.xlist[i];
    if (!in_range(r, 0, w.J, w.status)) continue;
    const int e = w.jend[r];
    const int p = Finish::active ? w.jparent[r] : -1;
    if (!in_range(e, r + 1, (long long)w.J + 1, w.status)) continue;
    const typename Finish::In x = fin.load(w, r, p, 0);
    const int t = r / JT;
    const int t2 = e / JT;
    V acc = M::load(out, r);
    acc = M::combine(acc, seg_fold_batched<M>(node, w.PJ, t + 1, t2 - 1));
    const int R2 = t2 * JT;
    if (e > R2) {
      const int c2 = (e - R2) / JC;
      const void* ct = static_cast<const unsigned char*>(w.ctree) +
                       (size_t)t2 * 2 * NCH * sizeof(V);
      auto cnode = [ct](int j) { return M::load(ct, j); };
      acc = M::combine(acc, seg_fold_batched<M>(cnode, NCH, 0, c2 - 1));
      // the joints of the end tile's chunk c2 before e (fewer than JC), from
      // their values: the fold over a range is the fold of its elements
      V vj[JC - 1];
#pragma unroll
      for (int q = 0; q < JC - 1; ++q) {
        const int j = R2 + c2 * JC + q;
        vj[q] = j < e ? values(j) : M::identity();
      }
#pragma unroll
      for (int q = 0; q < JC - 1; ++q) acc = M::combine(acc, vj[q]);
    }
    if (Finish::active) fin.apply(r, acc, x);
    else M::store(out, r, acc);
  }
}

}  // namespace tb

#endif  // TB_TREE_KERNELS_CUH
