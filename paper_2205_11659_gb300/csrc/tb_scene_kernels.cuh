// tb_scene_kernels.cuh -- kernels of the matching and bounding-box passes.
//
// The stream is cut into tiles of TILE elements; one block of NT threads
// owns a tile and each thread a chunk of KPT consecutive elements.
//
//   k1_tile_summary  one pass over the kind stream: per tile the bicyclic
//                    summary Bic(tile) = (a, b) (Sec. 3) and depth change,
//                    and the tile's stack slice (its unmatched opens,
//                    Sec. 7.1) with the running intersection of their clip
//                    boxes (Sec. 9).
//   k1_tile_prefix   one block: the global depth at every tile start (scan
//                    of the tiles' depth changes), the balance checks, and
//                    the min tree over the tiles' lowest depths.
//   k2_tile_resolve  the tile-level tree: for every tile the owner of the
//                    depth just below its slice (ps) and of the depth just
//                    below its start (q), found by the up/down tree search
//                    of Fig. "core" over a tree of tile minima; the owner
//                    segments of the stack at every tile start; then the
//                    clip in force below each slice by pointer jumping over
//                    the ps links (Sec. 6.1).
//   k3_tile          the main pass: reads kinds and boxes once, resolves
//                    every element's parent from its own chunk, an earlier
//                    chunk of the tile, or the tile context (the top of the
//                    stack at the tile start, Sec. 4: a close-only suffix
//                    indexes directly into a materialised stack slice),
//                    intersects leaves with their clip chain, and unions
//                    leaves up into every open whose close lies in the same
//                    tile (Sec. 6.2: descendants are a contiguous slice).
//   k4_*             unions of pairs whose open and close lie in different
//                    tiles, from per-tile partial unions and a union tree
//                    over tiles.
#ifndef TB_SCENE_KERNELS_CUH
#define TB_SCENE_KERNELS_CUH

#include <cooperative_groups.h>

#include "tb_core.cuh"

namespace tb {

// Loads the KPT kinds of a chunk starting at global index e0.  Positions at
// or past n read as K_PAD; in-range bytes above 3 are reported and then
// treated as leaves so that the pass stays well defined.
__device__ __forceinline__ bool load_kinds(const uint8_t* __restrict__ kind, int n, int e0,
                                           uint8_t (&kk)[KPT]) {
  bool bad = false;
  if (e0 + KPT <= n) {
    // one aligned vector load of the chunk's KPT bytes (e0 is a multiple of KPT)
    unsigned w[KPT / 4];
    if constexpr (KPT == 16) {
      const uint4 v = ld_nc_u4(kind + e0);
      w[0] = v.x;
      w[1] = v.y;
      w[2] = v.z;
      w[3] = v.w;
    } else if constexpr (KPT == 12) {  // e0 a multiple of 12: three aligned words
      const unsigned* q = reinterpret_cast<const unsigned*>(kind + e0);
      w[0] = __ldg(q);
      w[1] = __ldg(q + 1);
      w[2] = __ldg(q + 2);
    } else {
      const uint2 v = ld_nc_u2(kind + e0);
      w[0] = v.x;
      w[1] = v.y;
    }
#pragma unroll
    for (int i = 0; i < KPT; ++i) kk[i] = (uint8_t)((w[i >> 2] >> (8 * (i & 3))) & 0xffu);
#pragma unroll
    for (int i = 0; i < KPT; ++i)
      if (kk[i] > 3) { bad = true; kk[i] = K_LEAF; }
  } else {
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      if (e0 + i < n) {
        uint8_t k = kind[e0 + i];
        if (k > 3) { bad = true; k = K_LEAF; }
        kk[i] = k;
      } else {
        kk[i] = K_PAD;
      }
    }
  }
  return bad;
}

// The KPT kinds of a chunk as KPT/4 little-endian words of bytes (positions
// at or past n read as leaves; in-range bytes above 3 are reported and then
// treated as leaves, as load_kinds does).
__device__ __forceinline__ bool load_kind_words(const uint8_t* __restrict__ kind, int n, int e0,
                                                unsigned (&wd)[KPT / 4]) {
  bool bad = false;
  if (e0 + KPT <= n) {
    if constexpr (KPT == 16) {
      const uint4 v = ld_nc_u4(kind + e0);
      wd[0] = v.x;
      wd[1] = v.y;
      wd[2] = v.z;
      wd[3] = v.w;
    } else if constexpr (KPT == 12) {  // e0 a multiple of 12: three aligned words
      const unsigned* q = reinterpret_cast<const unsigned*>(kind + e0);
      wd[0] = __ldg(q);
      wd[1] = __ldg(q + 1);
      wd[2] = __ldg(q + 2);
    } else {
      const uint2 v = ld_nc_u2(kind + e0);
      wd[0] = v.x;
      wd[1] = v.y;
    }
#pragma unroll
    for (int j = 0; j < KPT / 4; ++j) {
      if (wd[j] & 0xfcfcfcfcu) {  // some byte above 3
        bad = true;
        unsigned x = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const unsigned k = (wd[j] >> (8 * b)) & 0xffu;
          x |= (k > 3u ? 0u : k) << (8 * b);
        }
        wd[j] = x;
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < KPT / 4; ++j) {
      unsigned x = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int e = e0 + 4 * j + b;
        unsigned k = e < n ? kind[e] : 0u;
        if (k > 3u) {
          bad = true;
          k = 0u;
        }
        x |= k << (8 * b);
      }
      wd[j] = x;
    }
  }
  return bad;
}

// Summary of 4 consecutive kinds (2 bits each in `code`, the first lowest)
// for the tile-summary pass, with P_e the depth after element e relative to
// the group start:
//   bits  0-3   P_3 + 4                 depth change
//   bits  4-7   min(0, P_0..P_3) + 4    lowest depth, the start included
//   bits  8-11  min(P_0..P_3) + 4       lowest depth after an element
//   bits 12-15  opens e with P_e <= P_q for every later q in the group
//               (unmatched inside the group: its final stack, P rising by one)
//   bits 16-19  P_e + 4 of the first of those
//   bits 20-23  clips
__host__ __device__ __forceinline__ constexpr unsigned k1_group_entry(unsigned code) {
  int P[4] = {0, 0, 0, 0};
  int p = 0, m0 = 0, ma = 4;
  unsigned clip = 0, opn = 0;
  for (int e = 0; e < 4; ++e) {
    const int k = (int)((code >> (2 * e)) & 3u);
    p += kind_delta(k);
    P[e] = p;
    m0 = m0 < p ? m0 : p;
    ma = ma < p ? ma : p;
    if (k == K_CLIP) clip |= 1u << e;
    if (kind_open(k)) opn |= 1u << e;
  }
  unsigned wm = 0;
  int l0 = 0, later = 4;
  for (int e = 3; e >= 0; --e) {
    if (((opn >> e) & 1u) && P[e] <= later) {
      wm |= 1u << e;
      l0 = P[e];
    }
    later = later < P[e] ? later : P[e];
  }
  return (unsigned)(p + 4) | (unsigned)(m0 + 4) << 4 | (unsigned)(ma + 4) << 8 | wm << 12 |
         (unsigned)(l0 + 4) << 16 | clip << 20;
}

// The 256 group summaries, computed by the compiler; the tile-summary pass
// reads them through the read-only path (one kilobyte, which stays in L1).
struct K1GroupTable {
  unsigned e[256];
};
__host__ __device__ constexpr K1GroupTable k1_group_table() {
  K1GroupTable g{};
  for (unsigned c = 0; c < 256; ++c) g.e[c] = k1_group_entry(c);
  return g;
}
static __device__ const K1GroupTable k1_gtab = k1_group_table();

// The 2-bit codes of a word's 4 kind bytes (each 0..3).
__device__ __forceinline__ unsigned kind_code4(unsigned w) {
  return (w & 0x3u) | ((w >> 6) & 0xcu) | ((w >> 12) & 0x30u) | ((w >> 18) & 0xc0u);
}

// ------------------------------------------------------------------- K1
struct K1Args {
  const uint8_t* kind;
  const float4* box;
  int n;
  SceneWs ws;
  int* status;
};

template <bool HAS_BOX>
__global__ void __launch_bounds__(NT, 4) k1_tile_summary(K1Args a) {
  __shared__ int s_scr[NW + 1];
  __shared__ int2 s_scr2[NW + 1];
  __shared__ float4 s_fscr[NW + 1];
  __shared__ int s_boff;
  const int tid = threadIdx.x;
  const int t = blockIdx.x;
  const int base = t * TILE, p0 = tid * KPT;

  unsigned wd[KPT / 4];
  if (load_kind_words(a.kind, a.n, base + p0, wd)) atomic_cas_i32(a.status, ST_OK, ST_BAD_KIND);

  // Chunk depth profile relative to the chunk start, 4 kinds at a time.
  unsigned ge[KPT / 4];
  int r = 0, mn = 0, mn_after = INT_MAX;
#pragma unroll
  for (int j = 0; j < KPT / 4; ++j) {
    ge[j] = __ldg(&k1_gtab.e[kind_code4(wd[j])]);  // the group summary (k1_group_entry)
    const int m0 = r + (int)((ge[j] >> 4) & 15u) - 4, ma = r + (int)((ge[j] >> 8) & 15u) - 4;
    mn = mn < m0 ? mn : m0;
    mn_after = mn_after < ma ? mn_after : ma;
    r += (int)(ge[j] & 15u) - 4;
  }
  // one scan gives the tile-relative depth at the chunk start and, in its
  // total, the tile's depth change and lowest depth
  int2 tot2;
  const int2 ex2 = block_excl_scan(make_int2(r, mn), make_int2(0, DEPTH_NONE), OpDepth(), s_scr2, &tot2);
  const int ds = ex2.x;  // tile-relative depth at chunk start
  const int tot = tot2.x;
  const int tile_lo = tot2.y;
  const int a_t = -tile_lo;  // Bic(tile).a: closes that pop below the tile start
  const int b_t = tot + a_t;  // Bic(tile).b: opens left unmatched at the tile end
  if (tid == 0) {
    a.ws.t_a[t] = a_t;
    a.ws.t_b[t] = b_t;
    a.ws.t_tot[t] = tot;
    // slots of the tile's slice in the open-side arrays, taken from a
    // counter (the order of the tiles' ranges does not matter); a balanced
    // stream needs at most slot_cap of them (every unmatched open has its
    // own close in a later tile), so running out means an unbalanced one
    int off = (int)atomic_add_u32(a.ws.counter + 2, (unsigned)b_t);
    if ((long long)off + b_t > a.ws.slot_cap) {
      atomic_cas_i32(a.status, ST_OK, ST_UNBALANCED);
      off = -1;
    }
    a.ws.t_boff[t] = off;
    s_boff = off;
  }
  const int suf_after = block_excl_suffix_min(ds + mn_after, s_scr);  // (its barriers publish s_boff)
  const int boff = s_boff;
  if (boff < 0) return;  // the same value for the whole block

  // The tile's stack slice: an open is unmatched in the tile when the depth
  // never comes back below its level before the tile ends.  Its slot is its
  // depth relative to the tile's lowest depth (Sec. 7.1).
  // Consecutive unmatched opens of a chunk sit one level apart (an open
  // between them that stayed open would be unmatched too), so the chunk's
  // slots are first_slot, first_slot + 1, ... in element order.
  // Per group (from the last): its opens unmatched inside it stay unmatched
  // in the tile while their depth is at most the lowest depth after the
  // group; they rise one level at a time, so they are the first n of them.
  unsigned umt = 0, clipm = 0;
  int first_slot = 0;
  {
    int suf = suf_after;
    int A = ds + r;  // depth at the end of group j
#pragma unroll
    for (int j = KPT / 4 - 1; j >= 0; --j) {
      const unsigned e = ge[j];
      const int As = A - ((int)(e & 15u) - 4);  // depth at the group start
      clipm |= ((e >> 20) & 15u) << (4 * j);
      const unsigned wm = (e >> 12) & 15u;
      if (wm) {
        const int l0 = (int)((e >> 16) & 15u) - 4;
        const int nw = popc(wm);
        const long long room = (long long)suf - As - l0 + 1;  // (suf may be INT_MAX)
        const int nsel = room < nw ? (int)room : nw;
        if (nsel > 0) {
          unsigned m = wm, sel = 0;
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (q < nsel) {
              sel |= m & (0u - m);
              m &= m - 1u;
            }
          umt |= sel << (4 * j);
          first_slot = As + l0 - 1 + a_t;
        }
      }
      const int ma = As + (int)((e >> 8) & 15u) - 4;
      suf = suf < ma ? suf : ma;
      A = As;
    }
  }
  int* slice_pos = a.ws.slice_pos + boff;
  {
    int slot = first_slot;
    for (unsigned m = umt; m; m &= m - 1, ++slot) slice_pos[slot] = base + p0 + lowest_set(m);
  }

  if (HAS_BOX) {
    // Running intersection along the slice (Sec. 9: the boxes of a stack
    // slice are the inclusive intersection scan of its clip boxes).
    float4 loc = box_universe();
    for (unsigned m = umt & clipm; m; m &= m - 1)
      loc = box_isect(loc, ld_nc_f4(a.box + base + p0 + lowest_set(m)));
    float4 tot4;
    float4 acc = block_excl_scan(loc, box_universe(), OpIsect(), s_fscr, &tot4);
    float4* slice_rel = a.ws.slice_rel + boff;
    int slot = first_slot;
    for (unsigned m = umt; m; m &= m - 1, ++slot) {
      const int i = lowest_set(m);
      if ((clipm >> i) & 1u) acc = box_isect(acc, ld_nc_f4(a.box + base + p0 + i));
      slice_rel[slot] = acc;
    }
  }
}

// Global depth at every tile start (Sec. 3: the tiles' bicyclic summaries
// combine in order; only their depth changes are needed here), in one block:
// an exclusive scan of the tiles' depth changes, the tiles' lowest depths,
// the balance checks, and the min tree over the lowest depths that the owner
// searches of the tile-level resolve use (leaves at [P, 2P), the ones past
// the last tile above any depth).  Warp w owns the leaves
// [w * span, (w + 1) * span) and walks them 32 at a time (coalesced); each
// such group's five lowest tree levels come from shuffles, the levels above
// from global memory while a level is wide, then from shared memory.
constexpr int NT2 = 1024;

__global__ void __launch_bounds__(NT2) k1_tile_prefix(SceneWs ws, int* status) {
  constexpr int NWP = NT2 / 32;
  __shared__ int s_w[NWP];
  __shared__ int s_wa[NWP];
  __shared__ int s_top[2 * NT2];
  const int T = ws.T, P = ws.P, tid = threadIdx.x, lane = lane_id(), wid = warp_id();
  int* tree = ws.lo_tree;
  const int LP = 31 - __clz(P);                 // P = 2^LP
  const int span = P / NWP > 32 ? P / NWP : 32;
  const int base = wid * span;
  const int rounds = base < P ? span / 32 : 0;  // warp-uniform
  // the warp's total depth change (RB rounds of loads in flight at a time)
  constexpr int RB = 4;
  int sum = 0, suma = 0;
  for (int r0 = 0; r0 < rounds; r0 += RB) {
#pragma unroll
    for (int k = 0; k < RB; ++k) {
      const int t = base + (r0 + k) * 32 + lane;
      if (r0 + k < rounds && t < T) {
        sum += __ldg(ws.t_tot + t);
        suma += __ldg(ws.t_a + t);
      }
    }
  }
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    sum += shfl_xor(sum, m);
    suma += shfl_xor(suma, m);
  }
  if (lane == 0) {
    s_w[wid] = sum;
    s_wa[wid] = suma;
  }
  __syncthreads();
  if (wid == 0) {
    const int v = s_w[lane];
    const int incl = warp_incl_scan(v, OpAdd());
    s_w[lane] = incl - v;  // exclusive prefix of the warps
    if (lane == NWP - 1 && incl != 0) atomic_cas_i32(status, ST_OK, ST_UNBALANCED);  // ends above 0
    const int va0 = s_wa[lane];
    s_wa[lane] = warp_incl_scan(va0, OpAdd()) - va0;
  }
  __syncthreads();
  int carry = s_w[wid];
  int carry_a = s_wa[wid];  // offsets of the tiles' unmatched closes in the close-side arrays
  bool bad = false;
  for (int r0 = 0; r0 < rounds; r0 += RB) {
    int vt[RB], va[RB];
#pragma unroll
    for (int k = 0; k < RB; ++k) {
      const int t = base + (r0 + k) * 32 + lane;
      const bool in = r0 + k < rounds && t < T;
      vt[k] = in ? __ldg(ws.t_tot + t) : 0;
      va[k] = in ? __ldg(ws.t_a + t) : 0;
    }
#pragma unroll
    for (int k = 0; k < RB; ++k) {
      if (r0 + k < rounds) {  // warp-uniform
        const int t = base + (r0 + k) * 32 + lane;
        const int incl = warp_incl_scan(vt[k], OpAdd());
        const int excl = carry + incl - vt[k];
        const int incla = warp_incl_scan(va[k], OpAdd());
        int v = 0x7f7f7f7f;  // past the last tile: above any depth
        if (t < T) {
          v = excl - va[k];
          ws.t_dstart[t] = excl;
          ws.t_lo[t] = v;
          ws.t_aoff[t] = carry_a + incla - va[k];
          bad |= v < 0;  // a close pops below the root
        }
        if (t < P) tree[P + t] = v;
        carry += shfl_idx(incl, 31);
        carry_a += shfl_idx(incla, 31);
#pragma unroll
        for (int l = 1; l <= 5; ++l) {
          v = min(v, shfl_xor(v, 1 << (l - 1)));
          if (l <= LP && (lane & ((1 << l) - 1)) == 0 && t < P) tree[(P + t) >> l] = v;
        }
      }
    }
  }
  if (bad) atomic_cas_i32(status, ST_OK, ST_UNBALANCED);
  __syncthreads();
  // Levels above the fifth: nodes [h, 2h) from [2h, 4h), in global memory
  // while a level has more nodes than half the block, then in shared memory.
  int h = P >> 6;
  for (; h > NT2 / 2; h >>= 1) {
    for (int i = h + tid; i < 2 * h; i += NT2) tree[i] = min(tree[2 * i], tree[2 * i + 1]);
    __syncthreads();
  }
  if (h >= 1) {
    for (int i = 2 * h + tid; i < 4 * h; i += NT2) s_top[i] = tree[i];  // i < 4h <= 2 * NT2
    __syncthreads();
    for (int g = h; g >= 1; g >>= 1) {
      for (int i = g + tid; i < 2 * g; i += NT2) s_top[i] = min(s_top[2 * i], s_top[2 * i + 1]);
      __syncthreads();
    }
    for (int i = 1 + tid; i < 2 * h; i += NT2) tree[i] = s_top[i];
  }
}

// ------------------------------------------------------------------- K2
// Tile-level resolve, one thread per tile.  lo_tree, the min tree over the
// tiles' lowest depths, was built by k1_tile_prefix.
constexpr int NTR = 256;

// Owner links: ps = owner of depth lo - 1 (last earlier tile whose lowest
// depth is at most lo - 1), q = owner of depth dstart - 1.
__global__ void __launch_bounds__(NTR) k2_links(SceneWs ws) {
  const int u = blockIdx.x * NTR + threadIdx.x;
  if (u >= ws.T || *ws.status != ST_OK) return;
  const int lo = ws.t_lo[u], ds = ws.t_dstart[u];
  ws.t_ps[u] = lo - 1 >= 0 ? tree_last_le(ws.lo_tree, ws.P, u, lo - 1) : -1;
  ws.t_q[u] = ds - 1 >= 0 ? tree_last_le(ws.lo_tree, ws.P, u, ds - 1) : -1;
}

// Owner segments of the stack at each tile start, depths ds-1 .. ds-1-a:
// from the owner q of depth ds-1, each owner covers down to its lowest depth
// and hands over to its ps.  With boxes, also the first step of the pointer
// jumping below: v(u) = relative clip of the ps tile's slice entry at depth
// lo(u)-1, link(u) = ps(u).
template <bool HAS_BOX>
__global__ void __launch_bounds__(NTR) k2_segments(SceneWs ws) {
  const int u = blockIdx.x * NTR + threadIdx.x;
  if (u >= ws.T || *ws.status != ST_OK) return;
  const int ds = ws.t_dstart[u];
  int dtop = ds - 1;
  const int dbot = ds - 1 - ws.t_a[u];
  int own = ws.t_q[u];
  int n = 0;
  int4* seg = ws.t_seg + (size_t)u * SEGK;
  while (dtop >= dbot && n < SEGK) {
    if (dtop < 0 || own < 0) {
      seg[n++] = make_int4(-1, 0, dbot, dtop);
      dtop = dbot - 1;
      break;
    }
    const int lo_o = ws.t_lo[own];
    const int lo_s = lo_o > dbot ? lo_o : dbot;
    ws.t_segb[(size_t)u * SEGK + n] = ws.t_boff[own] - lo_o;
    seg[n++] = make_int4(own, lo_o, lo_s, dtop);
    dtop = lo_s - 1;
    own = ws.t_ps[own];
  }
  if (dtop >= dbot) {
    ws.t_nseg[u] = SEGK + 1;
    ws.t_cont[u] = make_int2(own, dtop);
  } else {
    ws.t_nseg[u] = n;
  }
  if constexpr (HAS_BOX) {
    const int lo = ws.t_lo[u], p = ws.t_ps[u];
    float4 v = box_universe();
    int l = -1;
    if (lo - 1 >= 0 && p >= 0 && in_range(lo - 1 - ws.t_lo[p], 0, TILE, ws.status)) {
      v = ws.slice_rel[(size_t)ws.t_boff[p] + (lo - 1 - ws.t_lo[p])];
      l = p;
    }
    ws.t_val[0][u] = v;
    ws.t_link[0][u] = l;
  }
}

// B(u) = B(ps(u)) * v(u) is a fold along the ps chain: pointer jumping,
// each round doubling the covered chain length (Sec. 6.1), by all the
// blocks of a cooperative launch with a grid-wide barrier between rounds.
// `rounds` covers the longest possible chain (ceil(log2 T) + 1); the rounds
// after the chains have closed copy their values unchanged.  The link and
// value arrays are read past L1 (ld.cg): another block wrote them in the
// previous round.
constexpr int NTJ = 256;
__global__ void __launch_bounds__(NTJ) k2_jump(SceneWs ws, int rounds) {
  cooperative_groups::grid_group grid = cooperative_groups::this_grid();
  const int T = ws.T;
  if (*ws.status != ST_OK) return;  // no kernel running now writes it: the whole grid returns
  const int nthr = gridDim.x * NTJ;
  int cur = 0;
  for (int r = 0; r < rounds; ++r) {
    for (int u = blockIdx.x * NTJ + threadIdx.x; u < T; u += nthr) {
      const int l = __ldcg(ws.t_link[cur] + u);
      float4 v = __ldcg(ws.t_val[cur] + u);
      int nl = -1;
      if (l >= 0 && in_range(l, 0, T, ws.status)) {
        v = box_isect(__ldcg(ws.t_val[cur] + l), v);
        nl = __ldcg(ws.t_link[cur] + l);
      }
      __stcg(ws.t_val[cur ^ 1] + u, v);
      __stcg(ws.t_link[cur ^ 1] + u, nl);
    }
    cur ^= 1;
    grid.sync();
  }
  for (int u = blockIdx.x * NTJ + threadIdx.x; u < T; u += nthr) ws.t_B[u] = __ldcg(ws.t_val[cur] + u);
}

// ----------------------------------------------------- tile context helpers
// Source slot (tile * TILE + slot) of the stack entry at global depth gd,
// m = dstart - 1 - gd, at the start of tile t; -1 below the root.
__device__ __forceinline__ int ctx_src_of(const SceneWs& ws, int t, bool ovf, const int4* seg,
                                          int nseg, int gd, int m) {
  if (ovf) return (m >= 0 && m <= ws.t_a[t]) ? ws.ctx_src[(size_t)ws.t_aoff[t] + t + m] : -1;
  const int s = segk_find(seg, nseg, gd);
  if (s < 0 || seg[s].x < 0) return -1;
  return seg[s].x * TILE + (gd - seg[s].y);
}

// The stack entry at global depth gd, m = dstart - 1 - gd, at the start of
// tile t: its owner tile *u and its index *idx in the open-side arrays;
// false below the root.  segb holds the segments' index bases (t_segb).
__device__ __forceinline__ bool ctx_entry(const SceneWs& ws, int t, bool ovf, const int4* seg,
                                          const int* segb, int nseg, int gd, int m, int* u,
                                          long long* idx) {
  if (ovf) {
    const int src = ctx_src_of(ws, t, true, seg, nseg, gd, m);
    if (src < 0 || !in_range(src, 0, (long long)ws.T * TILE, ws.status)) return false;
    *u = src / TILE;
    *idx = slice_at(ws, src);
    return true;
  }
  const int s = segk_find(seg, nseg, gd);
  if (s < 0 || seg[s].x < 0) return false;
  *u = seg[s].x;
  const long long i = (long long)gd + segb[s];
  *idx = in_range(i, 0, ws.slot_cap, ws.status) ? i : 0;
  return true;
}

// For a tile whose owner chain has more than SEGK segments: writes the
// context sources of all `count` depths below the tile start into the
// tile's ctx_src row (the precomputed segments first, then the rest of the
// chain collected SEG_CAP segments at a time).
__device__ __forceinline__ void fill_ctx_overflow(SegState& S, const SceneWs& ws, int t,
                                                  int dstart, int count, const int4* seg) {
  const int tid = threadIdx.x;
  int* row = ws.ctx_src + (size_t)ws.t_aoff[t] + t;
  const int covered_lo = seg[SEGK - 1].z;
  for (int m = tid; m < count; m += NT) {
    const int d = dstart - 1 - m;
    if (d >= covered_lo) {
      const int s = segk_find(seg, SEGK, d);
      row[m] = (s >= 0 && seg[s].x >= 0) ? seg[s].x * TILE + (d - seg[s].y) : -1;
    }
  }
  if (tid == 0) {
    const int2 c = ws.t_cont[t];
    S.u = c.x;
    S.dtop = c.y;
    S.dbot = dstart - count;
  }
  __syncthreads();
  for (;;) {
    if (tid == 0) seg_collect(S, ws.t_ps, ws.t_lo, ws.status);
    __syncthreads();
    const int ns = S.n;
    const int hi = ns > 0 ? S.seg_hi[0] : 0, lo = ns > 0 ? S.seg_lo[ns - 1] : 1;
    for (int m = dstart - 1 - hi + tid; m <= dstart - 1 - lo; m += NT) {
      const int d = dstart - 1 - m;
      const int s = seg_find(S, d);
      const int u = s >= 0 ? S.seg_u[s] : -1;
      row[m] = u >= 0 ? u * TILE + (d - S.seg_ulo[s]) : -1;
    }
    const bool done = S.done;
    __syncthreads();
    if (done) break;
  }
}

// Min tree (or union tree) over the NT chunks, leaves at [NT, 2NT): the five
// lowest levels inside each warp by shuffles, the rest by warp 0.
template <class T, class Op>
__device__ __forceinline__ void build_chunk_tree(T* tree, T leaf, Op op) {
  const int tid = threadIdx.x, lane = lane_id();
  T v = leaf;
  tree[NT + tid] = v;
#pragma unroll
  for (int g = 2; g <= 32; g <<= 1) {
    v = op(v, shfl_xor(v, g >> 1));
    if ((lane & (g - 1)) == 0) tree[NT / g + tid / g] = v;
  }
  __syncthreads();
  if (tid < 32) {
    // NW warp nodes at [NW, 2NW): reduce them the same way
    T w = tid < NW ? tree[NW + tid] : tree[NW];
#pragma unroll
    for (int g = 2; g <= NW; g <<= 1) {
      w = op(w, shfl_xor(w, g >> 1));
      if (tid < NW && (tid & (g - 1)) == 0) tree[NW / g + tid / g] = w;
    }
  }
  __syncthreads();
}

// For the cross-chunk unions of the main pass, with two barriers: the
// lowest depth of the later chunks of the tile (*later_lo), the union of the
// later chunks' leaves (*rest), and the union tree over the chunks' leaf
// unions (leaves at [NT, 2NT)).  Inside each warp by shuffles, across the NW
// warps from their aggregates (s_wlo, s_wrun: NW + 1 entries each).
__device__ __forceinline__ void chunk_suffixes_and_union_tree(int lo, float4 run, float4* tree,
                                                              int* s_wlo, float4* s_wrun,
                                                              int* later_lo, float4* rest) {
  const int tid = threadIdx.x, lane = lane_id(), w = warp_id();
  int smin = lo;
  float4 sun = run;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = shfl_down(smin, d);
    const float4 yu = shfl_down(sun, d);
    if (lane + d < 32) {
      smin = smin < y ? smin : y;
      sun = box_unite(sun, yu);
    }
  }
  float4 v = run;
  tree[NT + tid] = v;
#pragma unroll
  for (int g = 2; g <= 32; g <<= 1) {
    v = box_unite(v, shfl_xor(v, g >> 1));
    if ((lane & (g - 1)) == 0) tree[NT / g + tid / g] = v;
  }
  if (lane == 0) {
    s_wlo[w] = smin;
    s_wrun[w] = sun;
  }
  __syncthreads();
  if (tid < 32) {
    // top of the union tree: NW warp nodes at [NW, 2NW)
    float4 x = tid < NW ? tree[NW + tid] : tree[NW];
#pragma unroll
    for (int g = 2; g <= NW; g <<= 1) {
      x = box_unite(x, shfl_xor(x, g >> 1));
      if (tid < NW && (tid & (g - 1)) == 0) tree[NW / g + tid / g] = x;
    }
    // exclusive suffix over the warps, in place (the warp after the last
    // holds the identities)
    if (tid == 0) {
      int am = INT_MAX;
      float4 au = box_empty();
      for (int i = NW - 1; i >= 0; --i) {
        const int xm = s_wlo[i];
        const float4 xu = s_wrun[i];
        s_wlo[i] = am;
        s_wrun[i] = au;
        am = am < xm ? am : xm;
        au = box_unite(xu, au);
      }
    }
  }
  __syncthreads();
  int exm = shfl_down(smin, 1);
  float4 exu = shfl_down(sun, 1);
  if (lane == 31) {
    exm = INT_MAX;
    exu = box_empty();
  }
  const int am = s_wlo[w];
  *later_lo = exm < am ? exm : am;
  *rest = box_unite(exu, s_wrun[w]);
}

// ------------------------------------------------------------------- K3
struct K3Args {
  const uint8_t* kind;
  const float4* box;
  int n;
  int32_t* parent;
  int32_t* match;
  float4* box_out;
  const int64_t* offsets;  // batched: scene offsets (num_scenes + 1)
  int num_scenes;
  int vec_out;             // parent/match are 16-byte aligned
  SceneWs ws;
  int* status;
  float4* clip_out;        // nullable: per element, the clip intersection in force (Sec. 9)
};

constexpr int CTXC = 32;      // top entries of the tile context cached in shared memory
constexpr int SOFF_CAP = 64;  // scene offsets of one tile staged in shared memory

// Dynamic shared memory of k3_tile.
__host__ __device__ constexpr int k3_smem_bytes(bool has_box) {
  return (has_box ? (BOX_SMEM_LEN * 16 + 2 * NT * 16 + NT * 16) : 0) + TILE * 4 + NT * 4 +
         2 * NT * 4 + NT * 4 + 2 * NT * 4;
}

// Fold of chunk-tree leaves l..r (inclusive); the loop has a fixed trip
// count and addresses that do not depend on loaded values.
template <class T, class Op>
__device__ __forceinline__ T chunk_range(const T* tree, int l, int r, T ident, Op op) {
  T left = ident, right = ident;
  if (l <= r) {
    l += NT;
    r += NT + 1;
#pragma unroll
    for (int lev = 0; lev <= 8; ++lev) {
      if (l < r) {
        if (l & 1) left = op(left, tree[l++]);
        if (r & 1) right = op(tree[--r], right);
      }
      l >>= 1;
      r >>= 1;
    }
  }
  return op(left, right);
}

// Where the stack entries below a chunk's own elements live: an earlier
// chunk of the tile (its slice in shared memory) or the tile context.
struct OutCtx {
  const int* s_lo;
  const int* s_cps;
  const int* s_spos;
  const float4* s_B;
  const float4* s_box;
  const int* s_cidx;
  const float4* s_cclip;
  const int4* s_seg;
  const int* s_segb;
  int nseg, ovf, t, dstart_t, base;
};
struct OutRes {
  int own, par;
  float4 cx;
};

// The entry at tile-relative depth dd of the stack at the start of the
// calling chunk: its global index and (want_clip) the clip in force there.
// `own` is the chunk cursor (owner of the previous, higher depth).
template <bool HAS_BOX>
__device__ __forceinline__ OutRes out_lookup(const OutCtx& c, const SceneWs& ws, int dd, int want_clip,
                                          int own) {
  OutRes r;
  r.cx = box_universe();
  while (own >= 0 && c.s_lo[own] > dd) own = c.s_cps[own];
  r.own = own;
  if (own >= 0) {
    const int si = own * KPT + (dd - c.s_lo[own]);
    const int op = in_range(si, 0, TILE, ws.status) ? c.s_spos[si] : 0;
    r.par = c.base + op;
    if (HAS_BOX && want_clip) r.cx = box_isect(c.s_B[own], c.s_box[box_slot(op)]);
  } else {
    const int m = -1 - dd;
    if (m < CTXC) {
      r.par = c.s_cidx[m];
      if (HAS_BOX && want_clip) r.cx = c.s_cclip[m];
    } else {
      int u;
      long long idx;
      const bool found = ctx_entry(ws, c.t, c.ovf != 0, c.s_seg, c.s_segb, c.nseg,
                                   c.dstart_t - 1 - m, m, &u, &idx);
      r.par = found ? ws.slice_pos[idx] : -1;
      if (HAS_BOX && want_clip && found) r.cx = box_isect(ws.t_B[u], ws.slice_rel[idx]);
    }
  }
  return r;
}

// One block per tile, or (TB_PERSIST) a grid of resident blocks that take
// tiles in order from a ticket counter (counter[1] of the workspace, zeroed
// at the start of each call), the next ticket drawn while the current tile is
// processed.  The per-tile code below is the same in both builds; it leaves a
// tile through K3_TILE_DONE (a return, or a break to the next ticket).  The
// matching-only pass is held to 64 registers a thread so that 1024 threads
// per SM stay resident.
// Blocks of the main pass that fit an SM together: five when a tile's box
// staging leaves room for them (at most 1536 elements: 42 KB of shared memory
// per block, and 96 registers per thread asked of the compiler), else two.
constexpr int K3_MIN_BLOCKS = TILE <= 1536 && NT == 128 ? 5 : 2;

template <bool HAS_BOX, bool BATCHED, bool CLIP = false>
__global__ void __launch_bounds__(NT, HAS_BOX ? K3_MIN_BLOCKS : 1024 / NT) k3_tile(K3Args a) {
  TB_DYNAMIC_SMEM(smem);
  __shared__ int s_scr[NW + 1];
  __shared__ int4 s_seg[SEGK];
  __shared__ int s_segb[SEGK];
  __shared__ int s_info[3];
  __shared__ int s_stop;
  __shared__ int s_cidx[CTXC];
  __shared__ float4 s_cclip[CTXC];
  __shared__ float4 s_fscr[NW];
  __shared__ SegState S;
  __shared__ long long s_soff[SOFF_CAP + 1];
  __shared__ int s_sc[2];

  const int tid = threadIdx.x;
#if TB_PERSIST
  __shared__ int s_next;
  if (tid == 0) s_next = (int)atomic_add_u32(a.ws.counter + 1, 1u);
  __syncthreads();
  for (int t = s_next; t < a.ws.T; t = s_next) {
    __syncthreads();  // every thread has read s_next
    if (tid == 0) s_next = (int)atomic_add_u32(a.ws.counter + 1, 1u);
    do {
#define K3_TILE_DONE break
#else
  {
    const int t = blockIdx.x;
#define K3_TILE_DONE return
#endif
  // ---- tile t
  const int base = t * TILE;
  const int cnt = min(TILE, a.n - base);
  const int p0 = tid * KPT;
  const SceneWs& ws = a.ws;
  // An error of the earlier passes leaves their tile data inconsistent: stop.
  // (This pass may itself report an unbalanced scene while other blocks run,
  // so one thread reads the word and the block follows it.)
  if (tid == 0) s_stop = *a.status;
  __syncthreads();
  if (s_stop != ST_OK) K3_TILE_DONE;

  unsigned char* sp = smem;
  float4* s_box = reinterpret_cast<float4*>(sp);
  float4* s_val = s_box + BOX_SMEM_LEN;  // 2*NT: pointer jumping, then the union tree
  float4* s_span = s_val + 2 * NT;       // NT: union of the chunks (cps(x), x]
  if (HAS_BOX) sp += BOX_SMEM_LEN * 16 + 2 * NT * 16 + NT * 16;
  int* s_spos = reinterpret_cast<int*>(sp);  // chunk slices; entries parked for the walk
  sp += TILE * 4;
  int* s_lo = reinterpret_cast<int*>(sp);
  sp += NT * 4;
  int* s_tree = reinterpret_cast<int*>(sp);
  sp += 2 * NT * 4;
  int* s_cps = reinterpret_cast<int*>(sp);
  sp += NT * 4;
  int* s_link = reinterpret_cast<int*>(sp);

  // ---- stage: tile info, kinds into registers, boxes into shared memory
  if (tid == 0) {
    s_info[0] = ws.t_a[t];
    s_info[1] = ws.t_dstart[t];
    s_info[2] = ws.t_nseg[t];
  }
  if (tid < SEGK) {
    s_seg[tid] = ws.t_seg[(size_t)t * SEGK + tid];
    s_segb[tid] = ws.t_segb[(size_t)t * SEGK + tid];
  }
  // The tile context's top CTXC entries are the longest chain of dependent
  // loads (tile info, owner segments, slice entry, clips): warp 0 issues them
  // first, reading the tile info and segments itself, so that they overlap
  // the kinds-only work below (a tile whose segment list overflowed takes
  // the slower path further down instead).
  int ctx_i = -1;
  float4 ctx_c = box_universe();
  bool ctx_early = false;
  if (tid < CTXC) {
    const int a0 = ws.t_a[t], d0 = ws.t_dstart[t], ns0 = ws.t_nseg[t];
    ctx_early = ns0 <= SEGK;
    if (ctx_early && tid <= a0) {
      const int gd = d0 - 1 - tid;
      int u = -1;
      long long si = 0;
      for (int i = 0; i < ns0; ++i) {
        const int4 sg = ws.t_seg[(size_t)t * SEGK + i];
        if (gd >= sg.z && gd <= sg.w) {
          u = sg.x;
          si = (long long)gd + ws.t_segb[(size_t)t * SEGK + i];
          break;
        }
      }
      if (u >= 0 && in_range(si, 0, ws.slot_cap, ws.status)) {
        ctx_i = ws.slice_pos[si];
        if (HAS_BOX) ctx_c = box_isect(ws.t_B[u], ws.slice_rel[si]);
      }
    }
  }
  if (BATCHED && tid < 2) {
    // scene of the tile's first (tid 0) and last (tid 1) element
    const int64_t e = base + (tid == 0 ? 0 : cnt - 1);
    int lo = 0, hi = a.num_scenes;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.offsets[mid] <= e) lo = mid; else hi = mid - 1;
    }
    s_sc[tid] = lo < a.num_scenes ? lo : a.num_scenes - 1;
  }
  uint8_t kk[KPT];
  load_kinds(a.kind, a.n, base + p0, kk);  // bad kinds were reported by k1
  if (HAS_BOX) {
    // asynchronous global -> shared copies; the kinds-only work below runs
    // while they are in flight
#pragma unroll 4
    for (int i = 0; i < KPT; ++i) {
      const int p = i * NT + tid;
      if (p < cnt) cp_async16(&s_box[box_slot(p)], a.box + base + p);
    }
    cp_async_commit();
  }

  // ---- in-chunk structure from the kinds alone (register stack of
  // 4-bit positions): parent position, partner position, masks.
  unsigned long long lpar = 0, lmate = 0;
  unsigned inside = 0, pairm = 0, openm = 0, closem = 0, clipm = 0;
  {
    unsigned long long stk = 0;
    int spn = 0;
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      const int k = kk[i];
      if (spn > 0) {
        inside |= 1u << i;
        lpar |= (stk & 15ull) << (4 * i);
      }
      if (k == K_CLIP || k == K_BLEND) {
        openm |= 1u << i;
        if (k == K_CLIP) clipm |= 1u << i;
        stk = (stk << 4) | (unsigned long long)i;
        ++spn;
      } else if (k == K_CLOSE) {
        closem |= 1u << i;
        if (spn > 0) {
          const int o = (int)(stk & 15ull);
          stk >>= 4;
          --spn;
          pairm |= (1u << i) | (1u << o);
          lmate |= ((unsigned long long)o << (4 * i)) | ((unsigned long long)i << (4 * o));
        }
      }
    }
  }
  const unsigned um = openm & ~pairm;   // the chunk's slice: opens unmatched in the chunk
  const unsigned xcl = closem & ~pairm;  // closes matching an open before the chunk
  const int a_j = popc(xcl);
  int tot;
  const int ds = block_excl_scan(popc(openm) - popc(closem), 0, OpAdd(), s_scr, &tot);
  const int lo_j = ds - a_j;
  s_lo[tid] = lo_j;
  // Chunk stack slice: the k-th unmatched open sits at depth lo_j + k.
  {
    int k = 0;
    for (unsigned m = um; m; m &= m - 1) s_spos[p0 + k++] = p0 + lowest_set(m);
  }
  const int a_t = s_info[0], dstart_t = s_info[1], nseg = s_info[2];
  const bool ovf = nseg > SEGK;
  // first close-side and open-side slots of the tile, read once (the stores
  // into the slot arrays would otherwise make the compiler reload them)
  const size_t aoff_t = (size_t)ws.t_aoff[t], boff_t = (size_t)ws.t_boff[t];

  // ---- tile context of a tile whose owner segments overflowed (the other
  // tiles loaded it at the start): the sources of every depth below the tile
  // start, then the top CTXC entries as above
  if (ovf) fill_ctx_overflow(S, ws, t, dstart_t, a_t + 1, s_seg);
  const bool ctx_mine = tid < CTXC && tid <= a_t;
  if (ctx_mine && !ctx_early) {
    int u;
    long long si;
    if (ctx_entry(ws, t, ovf, s_seg, s_segb, nseg, dstart_t - 1 - tid, tid, &u, &si)) {
      ctx_i = ws.slice_pos[si];
      if (HAS_BOX) ctx_c = box_isect(ws.t_B[u], ws.slice_rel[si]);
    }
  }

  if (ctx_mine) {
    s_cidx[tid] = ctx_i;
    if (HAS_BOX) s_cclip[tid] = ctx_c;
  }
  if (HAS_BOX) {
    cp_async_wait_all();
    __syncthreads();
    // Relative clip of each chunk-slice entry (intersection of the chunk's
    // unmatched clip boxes up to it), stored over that open's staged box.
    float4 acc = box_universe();
    for (unsigned m = um; m; m &= m - 1) {
      const int i = lowest_set(m);
      float4* b = &s_box[box_slot(p0 + i)];
      if ((clipm >> i) & 1u) acc = box_isect(acc, *b);
      *b = acc;
    }
  }
  build_chunk_tree(s_tree, lo_j, OpMin());

  // scene offsets of the tile
  int sc0 = 0;
  bool soff_smem = false;
  if (BATCHED) {
    sc0 = s_sc[0];
    const int nsc = s_sc[1] - s_sc[0] + 2;
    soff_smem = nsc <= SOFF_CAP + 1;
    if (soff_smem && tid < nsc) s_soff[tid] = a.offsets[sc0 + tid];
  }

  // ---- chunk links: cps = owner of depth lo_j - 1, cq = owner of ds - 1.
  // A tile-relative depth is owned by the last earlier chunk reaching down to
  // it (whatever its sign: chunks may pop below the tile start and push
  // again); with no such chunk it belongs to the tile context.
  const int cps = tree_last_le(s_tree, NT, tid, lo_j - 1);
  const int cq = tree_last_le(s_tree, NT, tid, ds - 1);
  s_cps[tid] = cps;  // published by the barrier below (with the jumping's first values)

  OutCtx oc;
  oc.s_lo = s_lo;
  oc.s_cps = s_cps;
  oc.s_spos = s_spos;
  oc.s_box = s_box;
  oc.s_cidx = s_cidx;
  oc.s_cclip = s_cclip;
  oc.s_seg = s_seg;
  oc.s_segb = s_segb;
  oc.nseg = nseg;
  oc.ovf = ovf;
  oc.t = t;
  oc.dstart_t = dstart_t;
  oc.base = base;

  int cur = 0;
  if (HAS_BOX) {
    // Clip in force below each chunk's slice: B(j) = B(cps) * v(j), folded
    // by pointer jumping (Sec. 6.1) with the tile context at the roots.
    float4 v;
    int link;
    if (cps >= 0) {
      v = s_box[box_slot(s_spos[cps * KPT + (lo_j - 1 - s_lo[cps])])];
      link = cps;
    } else {
      const int m = -lo_j;
      if (m < CTXC) {
        v = s_cclip[m];
      } else {
        int u;
        long long si;
        v = ctx_entry(ws, t, ovf, s_seg, s_segb, nseg, dstart_t - 1 - m, m, &u, &si)
                ? box_isect(ws.t_B[u], ws.slice_rel[si]) : box_universe();
      }
      link = -1;
    }
    s_val[tid] = v;
    s_link[tid] = link;
    __syncthreads();  // (also publishes s_cps)
    for (;;) {
      const int l = s_link[cur * NT + tid];
      float4 vv = s_val[cur * NT + tid];
      int nl = -1;
      if (l >= 0) {
        vv = box_isect(s_val[cur * NT + l], vv);
        nl = s_link[cur * NT + l];
      }
      s_val[(cur ^ 1) * NT + tid] = vv;
      s_link[(cur ^ 1) * NT + tid] = nl;
      const bool any = block_or(nl >= 0);
      cur ^= 1;
      if (!any) break;
    }
  }
  if (!HAS_BOX) __syncthreads();  // publishes s_cps
  oc.s_B = s_val + cur * NT;

  // ---- scene of the chunk's first element (batched)
  int64_t sc_start = 0, sc_next = INT64_MAX;
  int sc = 0;
  if (BATCHED) {
    const int64_t e0 = base + p0;
    if (soff_smem) {
      int lo = 0, hi = s_sc[1] - sc0;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_soff[mid] <= e0) lo = mid; else hi = mid - 1;
      }
      sc = sc0 + lo;
    } else {
      int lo = 0, hi = a.num_scenes;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.offsets[mid] <= e0) lo = mid; else hi = mid - 1;
      }
      sc = lo < a.num_scenes ? lo : a.num_scenes - 1;
    }
    sc_start = a.offsets[sc];
    sc_next = a.offsets[sc + 1];
  }
  const int64_t sc_start0 = sc_start, sc_next0 = sc_next;
  const int sc0c = sc;

  // ---- the stack entries below the chunk start that the chunk reaches:
  // entry m (m = 0 .. a_j) sits at tile-relative depth ds - 1 - m.  Entry 0
  // is the parent of the chunk's first elements at its base level; entry m
  // (m >= 1) becomes the parent of the base level after the chunk's m-th
  // unmatched close (which matches entry m - 1).  Entry 0 stays in
  // registers; for m >= 1 the index is parked in s_spos[p0 + KPT - m] (above
  // the chunk's slice: a_j + (slice length) <= KPT) and the clip in the box
  // slot of that m-th unmatched close (its own box is never read).  All
  // lookups run here, before the walk, so that the walk below has no
  // data-dependent loop.  (The slice entries and relative clips they read
  // are not written again until after the walk.)
  // An entry's clip is looked up only when an element other than an
  // unmatched close follows in its span, or when clip_out is written (an
  // unmatched close repeats the clip of the entry it closes).
  constexpr bool clip_all = HAS_BOX && CLIP;
  int par0;
  float4 clip0 = box_universe();
  {
    const OutRes r0 = out_lookup<HAS_BOX>(oc, ws, ds - 1, clip_all || !(xcl & 1u), cq);
    par0 = r0.par;
    clip0 = r0.cx;
    int own = r0.own;
    unsigned xm = xcl;
    for (int m = 1; m <= a_j; ++m) {
      const int c = lowest_set(xm);  // the m-th unmatched close
      xm &= xm - 1;
      const int want = clip_all || (c + 1 < KPT && !((xcl >> (c + 1)) & 1u));
      const OutRes r = out_lookup<HAS_BOX>(oc, ws, ds - 1 - m, want, own);
      own = r.own;
      s_spos[p0 + KPT - m] = r.par;
      if (HAS_BOX) s_box[box_slot(p0 + c)] = r.cx;
    }
  }

  // ---- the walk over the chunk's elements, the same instruction sequence
  // for every kind (selects and predicated shared-memory accesses instead of
  // branches, so that the lanes of a warp, whose elements differ in kind,
  // stay converged).  State: the clip in force (clip_top) and the union of
  // the leaves so far under the innermost open of the chunk (acc; at the
  // base level, all leaves of the chunk so far).  An open matched in the
  // chunk parks acc in its own box slot and the clip in force before it in
  // its close's slot; its close reads both back, writes the pair's union at
  // both ends and folds it into the restored acc.  An unmatched close keeps
  // the running union of the chunk's leaves in its slot (the part of its
  // pair's union that lies in this chunk) and takes the next entry parked
  // above.  An unmatched open also keeps acc in its slot (the leaves since
  // the previous unmatched open, or since the chunk start) and starts a new
  // acc; its clip is its relative clip, read from the same slot, meet the
  // clip in force.  Every slot is written with the same value, `own`, so
  // the store needs no select on the kind.  The other chunks' lookups above
  // read relative clips from those slots: the barrier first.
  __syncthreads();
  unsigned long long kpack = 0;  // kinds, 4 bits per element
#pragma unroll
  for (int i = 0; i < KPT; ++i) kpack |= (unsigned long long)kk[i] << (4 * i);
  int x_par = par0;   // parent of the base level
  int x_m = 0;        // unmatched closes so far
  float4 clip_top = clip0;
  float4 acc = box_empty();
  int D = ds;         // tile-relative depth before the current element (batched check)
  int4 pg = make_int4(-1, -1, -1, -1), mg = make_int4(-1, -1, -1, -1);
  const int bp0 = base + p0;
  // the next element's slot is loaded one element ahead; the only store of
  // an element that can hit the next slot is an open's parked clip when its
  // close follows at once, and that value is forwarded instead
  float4 bnext = box_universe();
  if (HAS_BOX) bnext = s_box[box_slot(p0)];
#pragma unroll 1
  for (int g = 0; g < KPT / 4; ++g) {
    // the group's 4-bit fields, so that the element loop below shifts by
    // compile-time amounts
    const unsigned gk = (unsigned)(kpack >> (16 * g)) & 0xffffu;
    const unsigned gpar = (unsigned)(lpar >> (16 * g)) & 0xffffu;
    const unsigned gmate = (unsigned)(lmate >> (16 * g)) & 0xffffu;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = 4 * g + q;
      const int k = (int)((gk >> (4 * q)) & 15u);
      const int p = p0 + i;
      const bool in_c = (inside >> i) & 1u;
      const bool pr = (pairm >> i) & 1u;
      const int lp = (int)((gpar >> (4 * q)) & 15u);
      const int pt = (int)((gmate >> (4 * q)) & 15u);
      const bool is_leaf = k == K_LEAF, is_close = k == K_CLOSE;
      const bool is_open = k == K_CLIP || k == K_BLEND;
      const bool is_uc = is_close && !pr;
      int par_i = in_c ? bp0 + lp : x_par;
      int mat_i = pr ? bp0 + pt : (is_close ? par_i : -1);
      if (HAS_BOX) {
        const int sp_own = box_slot(p), sp_pt = box_slot(p0 + pt);
        const float4 b = bnext;
        if (i + 1 < KPT) bnext = s_box[box_slot(p + 1)];
        const bool mc = is_close && pr;
        float4 r = box_empty();
        if (mc) r = s_box[sp_pt];  // acc parked by the open
        const float4 iv = box_isect(b, clip_top);
        const float4 lf = box_canon(iv);
        // the raw running intersection: own box meet the clip in force for a
        // leaf or clip open, the clip in force for a blend, the value of the
        // open it closes for a close (the clip in force inside that open)
        if (CLIP && k < K_PAD) a.clip_out[bp0 + i] = (is_leaf || k == K_CLIP) ? iv : clip_top;
        if (k < K_PAD) s_box[sp_own] = is_leaf ? lf : acc;
        if (pr) s_box[sp_pt] = is_open ? clip_top : acc;
        if (is_open && pr && pt == i + 1) bnext = clip_top;
        const float4 y = is_leaf ? lf : r;
        acc = is_open ? box_empty() : box_unite(acc, y);
        clip_top = (k == K_CLIP) ? iv : (is_close ? b : clip_top);
      }
      {
        // after an unmatched close the base level takes the next parked entry
        x_m += is_uc ? 1 : 0;
        const int nx = s_spos[p0 + KPT - (x_m > 0 ? x_m : 1)];
        x_par = is_uc ? nx : x_par;
      }
      if (BATCHED && k != K_PAD) {
        const int e = bp0 + i;
        while (e >= sc_next && sc < a.num_scenes - 1) {
          ++sc;
          sc_start = a.offsets[sc];
          sc_next = a.offsets[sc + 1];
        }
        if (e == sc_start && dstart_t + D != 0) atomic_cas_i32(a.status, ST_OK, ST_UNBALANCED);
        if (par_i >= 0) par_i = (int)(par_i - sc_start);
        if (mat_i >= 0) mat_i = (int)(mat_i - sc_start);
        D += kind_delta(k);
      }
      if (q == 0) { pg.x = par_i; mg.x = mat_i; }
      if (q == 1) { pg.y = par_i; mg.y = mat_i; }
      if (q == 2) { pg.z = par_i; mg.z = mat_i; }
      if (q == 3) { pg.w = par_i; mg.w = mat_i; }
    }
    // parent / match of four elements (opens matched outside the chunk get
    // -1 here; their close writes the real value later)
    const int e4 = bp0 + 4 * g;
    if (a.vec_out && e4 + 4 <= a.n) {
      if (a.parent) *reinterpret_cast<int4*>(a.parent + e4) = pg;
      if (a.match) *reinterpret_cast<int4*>(a.match + e4) = mg;
    } else {
      const int pa[4] = {pg.x, pg.y, pg.z, pg.w};
      const int ma[4] = {mg.x, mg.y, mg.z, mg.w};
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if (e4 + r < a.n) {
          if (a.parent) a.parent[e4 + r] = pa[r];
          if (a.match) a.match[e4 + r] = ma[r];
        }
      }
    }
  }

  __syncthreads();  // every walk has finished; relative clips are no longer read

  if (!HAS_BOX) {
    // Closes matching an open of an earlier chunk of this tile write that
    // open's match (after the owner's vector store above); closes matching an
    // open of an earlier tile leave it to the cross-tile pass.
    int u = cq;
    int64_t scs = sc_start0, scn = sc_next0;
    int scx = sc0c;
    unsigned m = xcl;
    while (m) {
      const int i = lowest_set(m);
      m &= m - 1;
      const unsigned below = (1u << i) - 1u;
      const int dd = ds + popc(openm & below) - popc(closem & below) - 1;
      const int e = base + p0 + i;
      if (BATCHED) {
        while (e >= scn && scx < a.num_scenes - 1) {
          ++scx;
          scs = a.offsets[scx];
          scn = a.offsets[scx + 1];
        }
      }
      const int eo = BATCHED ? (int)(e - scs) : e;
      while (u >= 0 && s_lo[u] > dd) u = s_cps[u];
      if (u >= 0) {
        const int si = u * KPT + (dd - s_lo[u]);
        if (a.match && in_range(si, 0, TILE, ws.status)) a.match[base + s_spos[si]] = eo;
      } else if (in_range(-1 - dd, 0, a_t, ws.status)) {
        ws.cpos[aoff_t + (-1 - dd)] = e;
        ws.cval[aoff_t + (-1 - dd)] = eo;
      }
    }
    K3_TILE_DONE;
  }

  // ---- unions across chunks (and the partial unions of cross-tile pairs)
  // Union of the chunk's leaves after each unmatched open (everything after
  // it in the chunk is inside it): the walk left in each unmatched open's
  // slot the leaves between it and the previous one (or the chunk start),
  // and acc holds the leaves after the last one; fold them from the back.
  // What remains is the union of all the chunk's leaves.
  float4 run = acc;
  for (unsigned m = um; m; m &= ~(1u << (31 - __clz(m)))) {
    float4* sl = &s_box[box_slot(p0 + 31 - __clz(m))];
    const float4 part = *sl;
    *sl = run;
    run = box_unite(part, run);
  }
  float4* s_ut = s_val;  // union tree over the chunks' leaf unions
  int later_lo;
  float4 rest;           // union of the later chunks' leaves
  chunk_suffixes_and_union_tree(lo_j, run, s_ut, s_scr, s_fscr, &later_lo, &rest);
  // span(x) = union of the chunks (cps(x), x]: what a close's union gains
  // when the entry it closes lies in the slice of the chunk below x's
  s_span[tid] = tree_range(s_ut, NT, cps + 1, tid, box_empty(), OpUnite());
  __syncthreads();
  {
    // Closes matching an open of an earlier chunk or tile; the m-th closes
    // entry m (its index parked above, entry 0's in par0): union = the open's
    // chunk after it + the whole chunks in between + this chunk before the
    // close (Sec. 6.2).  Entry m + 1 encloses entry m, so the unions nest and
    // accumulate: U(m+1) = U(m) + usuf(open m+1) + upre(close m+1), plus
    // span(owner of entry m) when the owner steps down a chunk (entry m sat
    // at the bottom of its chunk's slice, so the next owner is that chunk's
    // cps; below the tile start the tile's own leaves before the close are
    // all that is needed here).
    int64_t scs = sc_start0, scn = sc_next0;
    int scx = sc0c;
    float4 U = box_empty();
    int u_prev = -1;
    unsigned m_cl = xcl;
    for (int m = 0; m_cl; ++m) {
      const int i = lowest_set(m_cl);
      m_cl &= m_cl - 1;
      const int cp = p0 + i;
      const int e = base + cp;
      if (BATCHED) {
        while (e >= scn && scx < a.num_scenes - 1) {
          ++scx;
          scs = a.offsets[scx];
          scn = a.offsets[scx + 1];
        }
      }
      const int eo = BATCHED ? (int)(e - scs) : e;
      const int idx = m == 0 ? par0 : s_spos[p0 + KPT - m];
      const bool in_t = idx >= base && idx < base + TILE;
      const int u = in_t ? (idx - base) / KPT : -1;
      if (m == 0) U = tree_range(s_ut, NT, u + 1, tid - 1, box_empty(), OpUnite());
      else if (u != u_prev && in_range(u_prev, 0, NT, ws.status)) U = box_unite(U, s_span[u_prev]);
      U = box_unite(U, s_box[box_slot(cp)]);  // this chunk before the close
      if (in_t) {
        const int op = idx - base;
        U = box_unite(U, s_box[box_slot(op)]);  // the open's chunk after it
        s_box[box_slot(op)] = U;
        s_box[box_slot(cp)] = U;
        if (a.match) a.match[idx] = eo;
      } else if (in_range(m - ds, 0, a_t, ws.status)) {
        const size_t mm = aoff_t + (m - ds);  // below the tile start: k4 finishes the pair
        ws.upre[mm] = U;
        ws.cpos[mm] = e;
        ws.cval[mm] = eo;
      }
      u_prev = u;
    }
  }
  // Opens left unmatched at the tile end: union over the rest of the tile.
  {
    unsigned m = um;
    int dd = lo_j;
    while (m) {
      const int i = lowest_set(m);
      m &= m - 1;
      if (dd < later_lo)
        ws.usuf[boff_t + dd + a_t] = box_unite(s_box[box_slot(p0 + i)], rest);
      ++dd;
    }
  }
  if (tid == 0) ws.t_uall[t] = s_ut[1];
  __syncthreads();
#pragma unroll 4
  for (int i = 0; i < KPT; ++i) {
    const int p = i * NT + tid;
    if (p < cnt) a.box_out[base + p] = s_box[box_slot(p)];
  }
#if TB_PERSIST
    } while (0);
    __syncthreads();  // the next tile reuses the shared memory; s_next is set
  }
#else
  }
#endif
#undef K3_TILE_DONE
}

// ---------------------------------------------------- K3, search matcher
// The matching-only main pass as the paper's binary-search form (Sec. 5,
// Fig. "core"): instead of walking a stack per chunk, every element finds
// its parent by the up/down search over a tree of the tile's depths.  With
// d(p) the depth before element p (relative to the tile start), the parent
// of p is the last q < p with d(q) <= d(p) - 1 (the innermost open still
// open at p); a close's match is its parent, an open's match is written by
// its close.  When no such q lies in the tile the parent is the tile-context
// entry -d(p) (element 0 has depth 0, so then d(p) <= 0).  Single scenes
// only (the batched pass keeps the walk).  An alternative the autotuner
// builds and times (TB_MATCHER = 1), not the tuned default.
#ifndef TB_MATCHER
#define TB_MATCHER 0
#endif

__host__ __device__ constexpr int k3s_smem_bytes() { return 2 * TILE * 4; }
static_assert(TB_MATCHER != 1 || (TILE & (TILE - 1)) == 0,
              "the search matcher's min tree over a tile needs a power-of-two tile");

__global__ void __launch_bounds__(NT) k3_search(K3Args a) {
  TB_DYNAMIC_SMEM(smem);
  __shared__ int s_scr[NW + 1];
  __shared__ int s_cidx[CTXC];
  __shared__ int4 s_seg[SEGK];
  __shared__ int s_info[4];
  __shared__ SegState S;
  const int tid = threadIdx.x, t = blockIdx.x;
  const int base = t * TILE, cnt = min(TILE, a.n - base), p0 = tid * KPT;
  const SceneWs& ws = a.ws;
  int* s_tree = reinterpret_cast<int*>(smem);  // min tree of depths, leaves at [TILE, 2 TILE)
  if (tid == 0) {
    s_info[0] = ws.t_a[t];
    s_info[1] = ws.t_dstart[t];
    s_info[2] = ws.t_nseg[t];
    s_info[3] = *a.status;  // an error of the earlier passes: the block stops (below)
  }
  if (tid < SEGK) s_seg[tid] = ws.t_seg[(size_t)t * SEGK + tid];
  uint8_t kk[KPT];
  load_kinds(a.kind, a.n, base + p0, kk);
  int rel[KPT];
  int r = 0;
#pragma unroll
  for (int i = 0; i < KPT; ++i) {
    rel[i] = r;  // depth before element i, relative to the chunk start
    r += kk[i] == K_PAD ? 0 : kind_delta(kk[i]);
  }
  int tot;
  const int ds = block_excl_scan(r, 0, OpAdd(), s_scr, &tot);  // barriers: s_info visible
  const int a_t = s_info[0], dstart_t = s_info[1], nseg = s_info[2];
  if (s_info[3] != ST_OK) return;  // the same value for every thread: the whole block returns
  const bool ovf = nseg > SEGK;
#pragma unroll
  for (int i = 0; i < KPT; ++i)
    s_tree[TILE + p0 + i] = p0 + i < cnt ? ds + rel[i] : INT_MAX;
  if (ovf) fill_ctx_overflow(S, ws, t, dstart_t, a_t + 1, s_seg);
  if (tid < CTXC && tid <= a_t) {
    const int src = ctx_src_of(ws, t, ovf, s_seg, nseg, dstart_t - 1 - tid, tid);
    s_cidx[tid] = src >= 0 && in_range(src, 0, (long long)ws.T * TILE, ws.status) ? ws.slice_pos[slice_at(ws, src)] : -1;
  }
  __syncthreads();
  for (int h = TILE / 2; h >= 1; h >>= 1) {
    for (int i = h + tid; i < 2 * h; i += NT) s_tree[i] = min(s_tree[2 * i], s_tree[2 * i + 1]);
    __syncthreads();
  }
  // one element per thread and round, consecutive threads on consecutive
  // elements (coalesced stores)
  for (int i = 0; i < KPT; ++i) {
    const int p = i * NT + tid;
    if (p >= cnt) break;
    const int e = base + p;
    const int k = a.kind[e] > 3 ? K_LEAF : a.kind[e];
    const int d = s_tree[TILE + p];
    const int q = tree_last_le(s_tree, TILE, p, d - 1);
    int par;
    if (q >= 0) {
      par = base + q;
    } else {
      const int m = -d;  // tile-context entry of depth d - 1
      if (m < CTXC) {
        par = m <= a_t ? s_cidx[m] : -1;
      } else {
        const int src = ctx_src_of(ws, t, ovf, s_seg, nseg, dstart_t - 1 - m, m);
        par = src >= 0 && in_range(src, 0, (long long)ws.T * TILE, ws.status) ? ws.slice_pos[slice_at(ws, src)] : -1;
      }
    }
    a.parent[e] = par;
    a.match[e] = k == K_CLOSE ? par : -1;
  }
  __syncthreads();  // the opens' placeholders are written before their closes' matches
  for (int i = 0; i < KPT; ++i) {
    const int p = i * NT + tid;
    if (p >= cnt) break;
    const int e = base + p;
    if (a.kind[e] != K_CLOSE) continue;
    const int d = s_tree[TILE + p];
    const int q = tree_last_le(s_tree, TILE, p, d - 1);
    if (q >= 0) {
      a.match[base + q] = e;
    } else if (in_range(-d, 0, a_t, ws.status)) {
      ws.cpos[(size_t)ws.t_aoff[t] + (-d)] = e;
      ws.cval[(size_t)ws.t_aoff[t] + (-d)] = e;
    }
  }
}

// ------------------------------------------------------------------- K4
// Union table over the tiles' leaf unions (a sparse table: level k holds,
// for every tile u, the union of tiles u .. u + 2^k - 1, clamped at the last
// tile; level 0 is t_uall itself).  Union is idempotent, so the union of any
// tile range [l, r] is two entries of one level (overlapping halves): the
// cross-tile pass asks for one range per owner segment, with two
// independent loads instead of a walk up a tree.  Built level by level by
// all the blocks of a cooperative launch with a grid-wide barrier between
// levels (reads past L1, as in k2_jump).
constexpr int NTU = 256;
__global__ void __launch_bounds__(NTU) k4_union_table(SceneWs ws, int levels) {
  cooperative_groups::grid_group grid = cooperative_groups::this_grid();
  const int T = ws.T;
  if (*ws.status != ST_OK) return;  // no kernel running now writes it: the whole grid returns
  const int nthr = gridDim.x * NTU;
  const float4* prev = ws.t_uall;
  for (int k = 1; k < levels; ++k) {
    float4* cur = ws.uall_tree + (size_t)(k - 1) * T;
    const int half = 1 << (k - 1);
    for (int u = blockIdx.x * NTU + threadIdx.x; u < T; u += nthr) {
      const int v = u + half < T ? u + half : T - 1;
      __stcg(cur + u, box_unite(__ldcg(prev + u), __ldcg(prev + v)));
    }
    prev = cur;
    grid.sync();
  }
}

// Union of the tiles l .. r (empty box when l > r) from the union table.
__device__ __forceinline__ float4 tile_range_union(const SceneWs& ws, int l, int r) {
  if (l > r) return box_empty();
  const int k = 31 - __clz(r - l + 1);
  const float4* lev = k == 0 ? ws.t_uall : ws.uall_tree + (size_t)(k - 1) * ws.T;
  return box_unite(__ldcg(lev + l), __ldcg(lev + r - (1 << k) + 1));
}

struct K4Args {
  float4* box_out;
  int32_t* match;
  SceneWs ws;
};

// One block per tile with closes matching opens of earlier tiles: writes
// match[open] and, with boxes, the union at both ends of the pair.
template <bool HAS_BOX>
__global__ void __launch_bounds__(NT) k4_cross_tile_unions(K4Args a) {
  __shared__ int4 s_seg[SEGK];
  __shared__ int s_segb[SEGK];
  __shared__ float4 s_mid[SEGK];
  __shared__ int s_nseg;
  const SceneWs& ws = a.ws;
  const int t = blockIdx.x, tid = threadIdx.x;
  const int a_t = ws.t_a[t];
  if (a_t == 0 || *ws.status != ST_OK) return;
  const int dstart = ws.t_dstart[t];
  const size_t aoff_t = (size_t)ws.t_aoff[t];
  if (tid == 0) s_nseg = ws.t_nseg[t];
  if (tid < SEGK) {
    s_seg[tid] = ws.t_seg[(size_t)t * SEGK + tid];
    s_segb[tid] = ws.t_segb[(size_t)t * SEGK + tid];
  }
  __syncthreads();
  const int nseg = s_nseg;
  const bool ovf = nseg > SEGK;
  if (HAS_BOX && !ovf && tid < nseg) {
    const int u = s_seg[tid].x;
    s_mid[tid] = u >= 0 ? tile_range_union(ws, u + 1, t - 1) : box_empty();
  }
  __syncthreads();
  for (int m = tid; m < a_t; m += NT) {
    const int d = dstart - 1 - m;
    int u;
    long long si;
    if (!ctx_entry(ws, t, ovf, s_seg, s_segb, nseg, d, m, &u, &si)) continue;  // unbalanced input
    const int s = ovf ? -1 : segk_find(s_seg, nseg, d);
    const int o = ws.slice_pos[si];
    if (!in_range(o, 0, (long long)ws.T * TILE, ws.status)) continue;
    const size_t cm = aoff_t + m;
    if (a.match) a.match[o] = ws.cval[cm];
    if (HAS_BOX) {
      const float4 mid = ovf ? tile_range_union(ws, u + 1, t - 1) : s_mid[s];
      const int c = ws.cpos[cm];
      const float4 U = box_unite(box_unite(ws.usuf[si], mid), ws.upre[cm]);
      a.box_out[o] = U;
      if (in_range(c, 0, (long long)ws.T * TILE, ws.status)) a.box_out[c] = U;
    }
  }
}

}  // namespace tb

#endif  // TB_SCENE_KERNELS_CUH
