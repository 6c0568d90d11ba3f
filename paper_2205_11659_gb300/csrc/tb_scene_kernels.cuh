// tb_scene_kernels.cuh -- kernels of the matching and bounding-box passes.
//
// The stream is cut into tiles of TILE elements; one block of NT threads
// owns a tile and each thread a chunk of KPT consecutive elements.
//
//   k1_tile_summary  one pass over the kind stream: per tile the bicyclic
//                    summary Bic(tile) = (a, b) (Sec. 3), the global depth
//                    at the tile start by a decoupled look-back over the
//                    tiles' depth deltas, and the tile's stack slice (its
//                    unmatched opens, Sec. 7.1) with the running
//                    intersection of their clip boxes (Sec. 9).
//   k2_tile_resolve  the tile-level tree: for every tile the owner of the
//                    depth just below its slice (ps) and of the depth just
//                    below its start (q), found by the up/down tree search
//                    of Fig. "core" over a tree of tile minima; then the
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

#include "tb_core.cuh"

namespace tb {

// Loads the KPT kinds of a chunk starting at global index e0.  Positions at
// or past n read as K_PAD; in-range bytes above 3 are reported and then
// treated as leaves so that the pass stays well defined.
__device__ __forceinline__ bool load_kinds(const uint8_t* __restrict__ kind, int n, int e0,
                                           uint8_t (&kk)[KPT]) {
  bool bad = false;
  if (e0 + KPT <= n) {
    uint4 v = ld_nc_u4(kind + e0);
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
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

__device__ __forceinline__ unsigned long long lb_pack(unsigned flag, int v) {
  return ((unsigned long long)flag << 32) | (unsigned long long)(unsigned)v;
}

// ------------------------------------------------------------------- K1
struct K1Args {
  const uint8_t* kind;
  const float4* box;
  int n;
  SceneWs ws;
  int* status;
  int withhold;  // tile that never publishes (self-test of the bounded wait); -1 normally
};

template <bool HAS_BOX>
__global__ void __launch_bounds__(NT) k1_tile_summary(K1Args a) {
  __shared__ int s_scr[NW + 1];
  __shared__ float4 s_fscr[NW + 1];
  __shared__ int s_t, s_excl;
  const int tid = threadIdx.x;
  // Tiles are numbered in the order blocks start, so every tile a block
  // waits for belongs to a block that is already running.
  if (tid == 0) s_t = (int)atomic_add_u32(a.ws.counter, 1u);
  __syncthreads();
  const int t = s_t;
  const int base = t * TILE, p0 = tid * KPT;

  uint8_t kk[KPT];
  if (load_kinds(a.kind, a.n, base + p0, kk)) atomic_cas_i32(a.status, ST_OK, ST_BAD_KIND);

  // Chunk depth profile relative to the chunk start.
  int rr[KPT];
  int r = 0, mn = 0, mn_after = INT_MAX;
#pragma unroll
  for (int i = 0; i < KPT; ++i) {
    r += kind_delta(kk[i]);
    rr[i] = r;
    mn = mn < r ? mn : r;
    mn_after = mn_after < r ? mn_after : r;
  }
  int tot;
  const int ds = block_excl_scan(r, 0, OpAdd(), s_scr, &tot);  // tile-relative depth at chunk start
  const int lo_j = ds + mn;
  int tile_lo;
  block_excl_scan(lo_j, INT_MAX, OpMin(), s_scr, &tile_lo);
  const int a_t = -tile_lo;  // Bic(tile).a: closes that pop below the tile start
  const int b_t = tot + a_t;  // Bic(tile).b: opens left unmatched at the tile end
  const int suf_after = block_excl_suffix_min(ds + mn_after, s_scr);

  // Decoupled look-back (single pass) for the global depth at the tile
  // start: publish this tile's depth delta, then add predecessors' deltas
  // until one that already knows its inclusive prefix.
  if (tid == 0) {
    unsigned long long* lb = a.ws.lb;
    if (t != a.withhold) st_release_u64(lb + t, lb_pack(1u, tot));
    int excl = 0;
    bool timed_out = false;
    for (int j = t - 1; j >= 0; --j) {
      unsigned long long w;
      unsigned it = 0;
      for (;;) {
        w = ld_acquire_u64(lb + j);
        if ((w >> 32) != 0) break;
        if (++it >= SPIN_LIMIT) { timed_out = true; break; }
        poll_backoff(it);
      }
      if (timed_out) break;
      excl += (int)(unsigned)(w & 0xffffffffull);
      if ((w >> 32) == 2ull) break;
    }
    if (timed_out) atomic_cas_i32(a.status, ST_OK, ST_TIMEOUT);
    if (t != a.withhold) st_release_u64(lb + t, lb_pack(2u, excl + tot));
    s_excl = excl;
    a.ws.t_a[t] = a_t;
    a.ws.t_b[t] = b_t;
    a.ws.t_dstart[t] = excl;
    a.ws.t_lo[t] = excl - a_t;
    if (excl - a_t < 0) atomic_cas_i32(a.status, ST_OK, ST_UNBALANCED);
    if (t == a.ws.T - 1 && excl + tot != 0) atomic_cas_i32(a.status, ST_OK, ST_UNBALANCED);
  }

  // The tile's stack slice: an open is unmatched in the tile when the depth
  // never comes back below its level before the tile ends.  Its slot is its
  // depth relative to the tile's lowest depth (Sec. 7.1).
  unsigned umt = 0;
  {
    int suf = suf_after;
#pragma unroll
    for (int i = KPT - 1; i >= 0; --i) {
      const int A = ds + rr[i];
      suf = suf < A ? suf : A;
      if (kind_open(kk[i]) && A <= suf) umt |= 1u << i;
    }
  }
  int* slice_pos = a.ws.slice_pos + (size_t)t * TILE;
#pragma unroll
  for (int i = 0; i < KPT; ++i)
    if ((umt >> i) & 1u) slice_pos[ds + rr[i] - 1 + a_t] = base + p0 + i;

  if (HAS_BOX) {
    // Running intersection along the slice (Sec. 9: the boxes of a stack
    // slice are the inclusive intersection scan of its clip boxes).
    float4 loc = box_universe();
#pragma unroll
    for (int i = 0; i < KPT; ++i)
      if (((umt >> i) & 1u) && kk[i] == K_CLIP) loc = box_isect(loc, ld_nc_f4(a.box + base + p0 + i));
    float4 tot4;
    float4 acc = block_excl_scan(loc, box_universe(), OpIsect(), s_fscr, &tot4);
    float4* slice_rel = a.ws.slice_rel + (size_t)t * TILE;
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      if ((umt >> i) & 1u) {
        if (kk[i] == K_CLIP) acc = box_isect(acc, ld_nc_f4(a.box + base + p0 + i));
        slice_rel[ds + rr[i] - 1 + a_t] = acc;
      }
    }
  }
}

// ------------------------------------------------------------------- K2
constexpr int NT2 = 1024;

template <bool HAS_BOX>
__global__ void __launch_bounds__(NT2) k2_tile_resolve(SceneWs ws) {
  const int T = ws.T, P = ws.P, tid = threadIdx.x;
  int* tree = ws.lo_tree;
  for (int u = tid; u < P; u += NT2) tree[P + u] = u < T ? ws.t_lo[u] : INT_MAX;
  __syncthreads();
  for (int h = P >> 1; h >= 1; h >>= 1) {
    for (int i = h + tid; i < 2 * h; i += NT2) {
      const int l = tree[2 * i], r = tree[2 * i + 1];
      tree[i] = l < r ? l : r;
    }
    __syncthreads();
  }
  for (int u = tid; u < T; u += NT2) {
    const int lo = ws.t_lo[u], ds = ws.t_dstart[u];
    ws.t_ps[u] = lo - 1 >= 0 ? tree_last_le(tree, P, u, lo - 1) : -1;
    ws.t_q[u] = ds - 1 >= 0 ? tree_last_le(tree, P, u, ds - 1) : -1;
  }
  if (!HAS_BOX) return;
  __syncthreads();
  // v(u): relative clip of the ps tile's slice entry at depth lo(u)-1;
  // B(u) = B(ps(u)) * v(u) is then a fold along the ps chain, done by
  // pointer jumping: each round doubles the covered chain length.
  for (int u = tid; u < T; u += NT2) {
    const int lo = ws.t_lo[u], p = ws.t_ps[u];
    float4 v = box_universe();
    int l = -1;
    if (lo - 1 >= 0 && p >= 0) {
      v = ws.slice_rel[(size_t)p * TILE + (lo - 1 - ws.t_lo[p])];
      l = p;
    }
    ws.t_val[0][u] = v;
    ws.t_link[0][u] = l;
  }
  __syncthreads();
  int cur = 0;
  for (;;) {
    bool any = false;
    for (int u = tid; u < T; u += NT2) {
      const int l = ws.t_link[cur][u];
      float4 v = ws.t_val[cur][u];
      int nl = -1;
      if (l >= 0) {
        v = box_isect(ws.t_val[cur][l], v);
        nl = ws.t_link[cur][l];
      }
      ws.t_val[cur ^ 1][u] = v;
      ws.t_link[cur ^ 1][u] = nl;
      any |= nl >= 0;
    }
    any = block_or(any);
    cur ^= 1;
    if (!any) break;
  }
  for (int u = tid; u < T; u += NT2) ws.t_B[u] = ws.t_val[cur][u];
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
  SceneWs ws;
  int* status;
};

// Dynamic shared memory of k3_tile.
__host__ __device__ constexpr int k3_smem_bytes(bool has_box) {
  return (has_box ? (BOX_SMEM_LEN * 16 + 2 * NT * 16) : 0) + TILE * 2 + (TILE + 4) * 4 +
         NT * 4 + 2 * NT * 4 + NT * 4 + 2 * NT * 4;
}

// Fills s_ctx[m], m = 0 .. count-1, with the workspace slot (tile * TILE +
// slot) of the stack entry at global depth dstart-1-m in the stack at the
// start of tile t, or -1 below the root.
__device__ __forceinline__ void fill_tile_ctx(SegState& S, const SceneWs& ws, int t, int dstart,
                                              int count, int* s_ctx) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    S.u = ws.t_q[t];
    S.dtop = dstart - 1;
    S.dbot = dstart - count;
  }
  __syncthreads();
  for (;;) {
    if (tid == 0) seg_collect(S, ws.t_ps, ws.t_lo);
    __syncthreads();
    const int hi = S.seg_hi[0], lo = S.seg_lo[S.n - 1];
    for (int m = dstart - 1 - hi + tid; m <= dstart - 1 - lo; m += NT) {
      const int d = dstart - 1 - m;
      const int s = seg_find(S, d);
      const int u = s >= 0 ? S.seg_u[s] : -1;
      s_ctx[m] = u >= 0 ? u * TILE + (d - S.seg_ulo[s]) : -1;
    }
    const bool done = S.done;
    __syncthreads();
    if (done) break;
  }
}

template <bool HAS_BOX, bool BATCHED>
__global__ void __launch_bounds__(NT, 2) k3_tile(K3Args a) {
  TB_DYNAMIC_SMEM(smem);
  __shared__ int s_scr[NW + 1];
  __shared__ SegState S;

  const int tid = threadIdx.x;
  const int t = blockIdx.x;
  const int base = t * TILE;
  const int cnt = min(TILE, a.n - base);
  const int p0 = tid * KPT;
  const SceneWs& ws = a.ws;

  unsigned char* sp = smem;
  float4* s_box = reinterpret_cast<float4*>(sp);
  float4* s_val = s_box + BOX_SMEM_LEN;  // 2*NT: pointer jumping, then the union tree
  if (HAS_BOX) sp += BOX_SMEM_LEN * 16 + 2 * NT * 16;
  uint16_t* s_spos = reinterpret_cast<uint16_t*>(sp);
  sp += TILE * 2;
  int* s_ctx = reinterpret_cast<int*>(sp);
  sp += (TILE + 4) * 4;
  int* s_lo = reinterpret_cast<int*>(sp);
  sp += NT * 4;
  int* s_tree = reinterpret_cast<int*>(sp);
  sp += 2 * NT * 4;
  int* s_cps = reinterpret_cast<int*>(sp);
  sp += NT * 4;
  int* s_link = reinterpret_cast<int*>(sp);

  // ---- stage: kinds into registers, boxes into shared memory (coalesced)
  uint8_t kk[KPT];
  load_kinds(a.kind, a.n, base + p0, kk);  // bad kinds were reported by k1
  if (HAS_BOX) {
#pragma unroll 4
    for (int i = 0; i < KPT; ++i) {
      const int p = i * NT + tid;
      if (p < cnt) s_box[box_slot(p)] = ld_nc_f4(a.box + base + p);
    }
  }
  const int a_t = ws.t_a[t];
  const int dstart_t = ws.t_dstart[t];

  // ---- chunk summaries: Bic(chunk) = (a_j, b_j) and depth at chunk start
  int r = 0, mn = 0;
#pragma unroll
  for (int i = 0; i < KPT; ++i) {
    r += kind_delta(kk[i]);
    mn = mn < r ? mn : r;
  }
  const int a_j = -mn;
  int tot;
  const int ds = block_excl_scan(r, 0, OpAdd(), s_scr, &tot);  // tile-relative
  const int lo_j = ds - a_j;
  s_lo[tid] = lo_j;
  s_tree[NT + tid] = lo_j;

  // Chunk stack slice: the chunk's unmatched opens, slot = depth - lo_j.
  unsigned um = 0;
  {
    int rr[KPT];
    int x = 0;
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      x += kind_delta(kk[i]);
      rr[i] = x;
    }
    int suf = INT_MAX;
#pragma unroll
    for (int i = KPT - 1; i >= 0; --i) {
      suf = suf < rr[i] ? suf : rr[i];
      if (kind_open(kk[i]) && rr[i] <= suf) {
        um |= 1u << i;
        s_spos[p0 + rr[i] - 1 + a_j] = (uint16_t)(p0 + i);
      }
    }
  }
  __syncthreads();
  if (HAS_BOX) {
    // Relative clip of each chunk-slice entry (intersection of the chunk's
    // unmatched clip boxes up to it), stored over that open's staged box.
    float4 acc = box_universe();
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      if ((um >> i) & 1u) {
        float4* b = &s_box[box_slot(p0 + i)];
        if (kk[i] == K_CLIP) acc = box_isect(acc, *b);
        *b = acc;
      }
    }
  }
  // Min tree over the chunks' lowest depths.
  for (int h = NT >> 1; h >= 1; h >>= 1) {
    if (tid < h) {
      const int l = s_tree[2 * (h + tid)], rgt = s_tree[2 * (h + tid) + 1];
      s_tree[h + tid] = l < rgt ? l : rgt;
    }
    __syncthreads();
  }

  // ---- tile context: sources of the top a_t + 1 stack entries
  fill_tile_ctx(S, ws, t, dstart_t, a_t + 1, s_ctx);

  // ---- chunk links: cps = owner of depth lo_j - 1, cq = owner of ds - 1.
  // A tile-relative depth is owned by the last earlier chunk reaching down to
  // it (whatever its sign: chunks may pop below the tile start and push
  // again); with no such chunk it belongs to the tile context.
  const int cps = tree_last_le(s_tree, NT, tid, lo_j - 1);
  const int cq = tree_last_le(s_tree, NT, tid, ds - 1);
  s_cps[tid] = cps;

  int cur = 0;
  float4 Bx = box_universe();
  if (HAS_BOX) {
    // Clip in force below each chunk's slice: B(j) = B(cps) * v(j), folded
    // by pointer jumping (Sec. 6.1) with the tile context at the roots.
    float4 v;
    int link;
    const int dl = lo_j - 1;
    if (cps >= 0) {
      const int slot = dl - s_lo[cps];
      v = s_box[box_slot(s_spos[cps * KPT + slot])];
      link = cps;
    } else {
      const int src = s_ctx[-1 - dl];
      v = src >= 0 ? box_isect(ws.t_B[src / TILE], ws.slice_rel[src]) : box_universe();
      link = -1;
    }
    s_val[tid] = v;
    s_link[tid] = link;
    __syncthreads();
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
    Bx = s_val[cur * NT + tid];
  } else {
    __syncthreads();
  }
  const float4* s_B = s_val + cur * NT;

  // ---- scene bookkeeping (batched): scene of the chunk's first element
  int64_t sc_start = 0, sc_next = INT64_MAX;
  int sc = 0;
  if (BATCHED) {
    const int64_t e0 = base + p0;
    int lo = 0, hi = a.num_scenes;  // last s with offsets[s] <= e0
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.offsets[mid] <= e0) lo = mid; else hi = mid - 1;
    }
    sc = lo < a.num_scenes ? lo : a.num_scenes - 1;
    sc_start = a.offsets[sc];
    sc_next = a.offsets[sc + 1];
  }

  // ---- the walk: one pass over the chunk with a local stack
  int D = ds;          // tile-relative depth before the current element
  int own = cq;        // chunk owning depth D-1 while the local stack is empty
  uint8_t st_pos[KPT];
  float4 st_acc[KPT];
  int sp_n = 0;
  float4 top_clip = box_universe();
  float4 cur_acc = box_empty();
  float4 run = box_empty();  // union of all leaf boxes of the chunk so far
  uint8_t xc_i[KPT];
  int xc_d[KPT];
  int nxc = 0;
  int32_t* const parent = a.parent;
  int32_t* const match = a.match;

  for (int i = 0; i < KPT; ++i) {
    const int k = kk[i];
    if (k == K_PAD) break;
    const int p = p0 + i;
    const int e = base + p;
    if (BATCHED) {
      while (e >= sc_next) {
        ++sc;
        sc_start = a.offsets[sc];
        sc_next = a.offsets[sc + 1];
      }
      if (e == sc_start && dstart_t + D != 0) atomic_cas_i32(a.status, ST_OK, ST_UNBALANCED);
    }
    // Parent and clip context: the local top, else the entry at depth D-1
    // of the stack at the chunk start.
    int par;
    float4 ctx = box_universe();
    if (sp_n > 0) {
      par = base + p0 + st_pos[sp_n - 1];
      ctx = top_clip;
    } else {
      const int dd = D - 1;
      while (own >= 0 && s_lo[own] > dd) own = s_cps[own];
      if (own >= 0) {
        const int op = s_spos[own * KPT + (dd - s_lo[own])];
        par = base + op;
        if (HAS_BOX) ctx = box_isect(s_B[own], s_box[box_slot(op)]);
      } else {
        const int src = s_ctx[-1 - dd];
        par = src >= 0 ? ws.slice_pos[src] : -1;
        if (HAS_BOX && src >= 0) ctx = box_isect(ws.t_B[src / TILE], ws.slice_rel[src]);
      }
    }
    const int par_out = (BATCHED && par >= 0) ? (int)(par - sc_start) : par;
    const int e_out = BATCHED ? (int)(e - sc_start) : e;
    if (k == K_LEAF) {
      if (parent) parent[e] = par_out;
      if (match) match[e] = -1;
      if (HAS_BOX) {
        float4* b = &s_box[box_slot(p)];
        const float4 out = box_canon(box_isect(*b, ctx));
        *b = out;
        run = box_unite(run, out);
        if (sp_n > 0) cur_acc = box_unite(cur_acc, out);
      }
    } else if (k == K_CLIP || k == K_BLEND) {
      if (parent) parent[e] = par_out;
      float4 clip = ctx;
      if (HAS_BOX) {
        float4* b = &s_box[box_slot(p)];
        if ((um >> i) & 1u) {
          clip = box_isect(Bx, *b);  // chunk-slice entry: B(j) * relative clip
        } else {
          if (k == K_CLIP) clip = box_isect(ctx, *b);
          *b = clip;  // kept for when this open is the top again
        }
      }
      if (sp_n > 0) st_acc[sp_n - 1] = cur_acc;
      st_pos[sp_n++] = (uint8_t)i;
      cur_acc = box_empty();
      top_clip = clip;
      ++D;
    } else {  // close
      if (sp_n > 0) {
        const int oi = st_pos[--sp_n];
        const int o = base + p0 + oi;
        const int o_out = BATCHED ? (int)(o - sc_start) : o;
        if (parent) parent[e] = o_out;
        if (match) {
          match[e] = o_out;
          match[o] = e_out;
        }
        if (HAS_BOX) {
          const float4 U = cur_acc;
          s_box[box_slot(p0 + oi)] = U;
          s_box[box_slot(p)] = U;
          if (sp_n > 0) {
            cur_acc = box_unite(st_acc[sp_n - 1], U);
            const int ti = st_pos[sp_n - 1];
            const float4 tb = s_box[box_slot(p0 + ti)];
            top_clip = ((um >> ti) & 1u) ? box_isect(Bx, tb) : tb;
          } else {
            cur_acc = box_empty();
          }
        }
      } else {
        // Matches an open before the chunk: the context entry at depth D-1.
        if (parent) parent[e] = par_out;
        if (match) {
          match[e] = par_out;
          if (par >= 0) match[par] = e_out;
        }
        if (HAS_BOX) s_box[box_slot(p)] = run;  // leaves of the chunk before it
        xc_i[nxc] = (uint8_t)i;
        xc_d[nxc] = D - 1;
        ++nxc;
      }
      --D;
    }
  }

  if (!HAS_BOX) return;

  // Unions of the opens still on the local stack over the rest of the
  // chunk: fold from the top down.
  {
    float4 u = box_empty();
    for (int s = sp_n - 1; s >= 0; --s) {
      const float4 acc_s = (s == sp_n - 1) ? cur_acc : st_acc[s];
      u = box_unite(acc_s, u);
      st_acc[s] = u;
    }
  }
  __syncthreads();  // every walk has finished reading relative clips
  for (int s = 0; s < sp_n; ++s) s_box[box_slot(p0 + st_pos[s])] = st_acc[s];
  float4* s_ut = s_val;  // union tree over the chunks' leaf unions
  s_ut[NT + tid] = run;
  __syncthreads();
  for (int h = NT >> 1; h >= 1; h >>= 1) {
    if (tid < h) s_ut[h + tid] = box_unite(s_ut[2 * (h + tid)], s_ut[2 * (h + tid) + 1]);
    __syncthreads();
  }

  // Closes matching an open of an earlier chunk: union = the open's chunk
  // after it + whole chunks in between + this chunk before the close.
  {
    int u = cq;
    for (int c = 0; c < nxc; ++c) {
      const int cp = p0 + xc_i[c];
      const int dd = xc_d[c];
      const float4 upre = s_box[box_slot(cp)];
      while (u >= 0 && s_lo[u] > dd) u = s_cps[u];
      if (u >= 0) {
        const int op = s_spos[u * KPT + (dd - s_lo[u])];
        const float4 mid = tree_range(s_ut, NT, u + 1, tid - 1, box_empty(), OpUnite());
        const float4 U = box_unite(box_unite(s_box[box_slot(op)], mid), upre);
        s_box[box_slot(op)] = U;
        s_box[box_slot(cp)] = U;
      } else {
        const int m = -1 - dd;
        const float4 mid = tree_range(s_ut, NT, 0, tid - 1, box_empty(), OpUnite());
        ws.upre[(size_t)t * TILE + m] = box_unite(mid, upre);
        ws.cpos[(size_t)t * TILE + m] = base + cp;
      }
    }
  }
  // Opens left unmatched at the tile end: union over the rest of the tile.
  if (sp_n > 0) {
    const int later_lo = tree_range(s_tree, NT, tid + 1, NT - 1, INT_MAX, OpMin());
    const float4 rest = tree_range(s_ut, NT, tid + 1, NT - 1, box_empty(), OpUnite());
    for (int s = 0; s < sp_n; ++s) {
      const int dd = lo_j + s;
      if (dd < later_lo) ws.usuf[(size_t)t * TILE + dd + a_t] = box_unite(st_acc[s], rest);
    }
  }
  if (tid == 0) ws.t_uall[t] = s_ut[1];
  __syncthreads();
#pragma unroll 4
  for (int i = 0; i < KPT; ++i) {
    const int p = i * NT + tid;
    if (p < cnt) a.box_out[base + p] = s_box[box_slot(p)];
  }
}

// ------------------------------------------------------------------- K4
__global__ void __launch_bounds__(NT2) k4_union_tree(SceneWs ws) {
  const int T = ws.T, P = ws.P, tid = threadIdx.x;
  float4* tree = ws.uall_tree;
  for (int u = tid; u < P; u += NT2) tree[P + u] = u < T ? ws.t_uall[u] : box_empty();
  __syncthreads();
  for (int h = P >> 1; h >= 1; h >>= 1) {
    for (int i = h + tid; i < 2 * h; i += NT2) tree[i] = box_unite(tree[2 * i], tree[2 * i + 1]);
    __syncthreads();
  }
}

struct K4Args {
  float4* box_out;
  SceneWs ws;
};

__global__ void __launch_bounds__(NT) k4_cross_tile_unions(K4Args a) {
  __shared__ SegState S;
  __shared__ float4 s_mid[SEG_CAP];
  const SceneWs& ws = a.ws;
  const int t = blockIdx.x, tid = threadIdx.x;
  const int a_t = ws.t_a[t];
  if (a_t == 0) return;
  const int dstart = ws.t_dstart[t];
  if (tid == 0) {
    S.u = ws.t_q[t];
    S.dtop = dstart - 1;
    S.dbot = dstart - a_t;
  }
  __syncthreads();
  for (;;) {
    if (tid == 0) seg_collect(S, ws.t_ps, ws.t_lo);
    __syncthreads();
    if (tid < S.n) {
      const int u = S.seg_u[tid];
      s_mid[tid] = u >= 0 ? tree_range(ws.uall_tree, ws.P, u + 1, t - 1, box_empty(), OpUnite())
                          : box_empty();
    }
    __syncthreads();
    const int hi = S.seg_hi[0], lo = S.seg_lo[S.n - 1];
    for (int m = dstart - 1 - hi + tid; m <= dstart - 1 - lo; m += NT) {
      const int d = dstart - 1 - m;
      const int s = seg_find(S, d);
      const int u = s >= 0 ? S.seg_u[s] : -1;
      if (u < 0) continue;
      const int src = u * TILE + (d - S.seg_ulo[s]);
      const int o = ws.slice_pos[src];
      const int c = ws.cpos[(size_t)t * TILE + m];
      const float4 U = box_unite(box_unite(ws.usuf[src], s_mid[s]), ws.upre[(size_t)t * TILE + m]);
      a.box_out[o] = U;
      a.box_out[c] = U;
    }
    const bool done = S.done;
    __syncthreads();
    if (done) break;
  }
}

}  // namespace tb

#endif  // TB_SCENE_KERNELS_CUH
