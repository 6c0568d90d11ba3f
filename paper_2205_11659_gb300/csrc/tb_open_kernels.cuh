// tb_open_kernels.cuh -- stream compaction of the opens: the stream index of
// every OPEN_CLIP / OPEN_BLEND element, in stream order.  A renderer keeps
// just the clip and blend nodes of a scene this way (Sec. 1.1), and position
// r of the result is the element of joint r in the tree scans.
//
// Reduce, scan, scatter over tiles of OTILE = 16384 elements:
//   k_open_count    per tile: number of opens (byte-parallel on 16-byte
//                   vectors); reports bytes above 3
//   k_open_offsets  one block: exclusive scan of the tile counts and the
//                   total
//   k_open_scatter  per tile: the positions in stream order, staged in
//                   shared memory and copied out coalesced
// The kinds are read twice (1 byte per element each time); the second read
// finds part of a large stream still in L2.
#ifndef TB_OPEN_KERNELS_CUH
#define TB_OPEN_KERNELS_CUH

#include "tb_core.cuh"

namespace tb {

// Compaction tiles: ONT threads, each with OVEC 16-byte vectors of kinds.
// Vector r of thread tid covers elements [r * ONT * 16 + tid * 16, +16) of
// the tile, so every round of loads is one contiguous, coalesced sweep.
constexpr int ONT = 256;
constexpr int ONW = ONT / 32;
constexpr int OVEC = 4;
constexpr int OROUND = ONT * 16;     // elements per round of vectors
constexpr int OTILE = OROUND * OVEC;  // elements per tile
constexpr int NTO = 1024;             // threads of the one-block offset scan

// Opens among the 16 kinds at global index e0 (bit i for element e0 + i;
// positions at or past n count as none).  *bad is set when an in-range byte
// is above 3; such bytes count as leaves.
__device__ __forceinline__ unsigned vec_open_mask(const uint8_t* __restrict__ kind, int n, int e0,
                                                  bool* bad) {
  unsigned m = 0, hi = 0;
  if (e0 + 16 <= n) {
    const uint4 v = ld_nc_u4(kind + e0);  // e0 is a multiple of 16
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      hi |= w[j] & 0xfcfcfcfcu;
      // kinds 1 and 2 are the bytes whose two low bits differ
      const unsigned f = (w[j] ^ (w[j] >> 1)) & 0x01010101u;
      // gather the four byte flags (bits 0, 8, 16, 24) into bits 21..24:
      // the shifted copies of the product never overlap, so nothing carries
      m |= ((f * 0x00204081u) >> 21 & 0xfu) << (4 * j);
    }
    if (hi != 0u) {  // bytes above 3 count as leaves
      m = 0;
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (kind_open((int)((w[i >> 2] >> (8 * (i & 3))) & 0xffu))) m |= 1u << i;
    }
  } else {
    for (int i = 0; i < 16; ++i) {
      if (e0 + i < n) {
        const unsigned k = kind[e0 + i];
        if (kind_open((int)k)) m |= 1u << i;
        hi |= k & ~3u;
      }
    }
  }
  *bad = hi != 0u;
  return m;
}

__global__ void __launch_bounds__(ONT) k_open_count(const uint8_t* __restrict__ kind, int n,
                                                    int* __restrict__ t_cnt, int* status) {
  __shared__ int s_scr[ONW + 1];
  const int t = blockIdx.x, tid = threadIdx.x;
  const int e0 = t * OTILE + tid * 16;
  unsigned m[OVEC];
  bool bad = false;
#pragma unroll
  for (int r = 0; r < OVEC; ++r) {
    bool b;
    m[r] = vec_open_mask(kind, n, e0 + r * OROUND, &b);
    bad |= b;
  }
  if (bad) atomic_cas_i32(status, ST_OK, ST_BAD_KIND);
  int c = 0;
#pragma unroll
  for (int r = 0; r < OVEC; ++r) c += popc(m[r]);
  int tot;
  block_excl_scan<ONW>(c, 0, OpAdd(), s_scr, &tot);
  if (tid == 0) t_cnt[t] = tot;
}

// t_off[t] = opens before tile t; *count = all opens.  Each round scans
// 4 * NTO tile counts, four per thread (one 16-byte load and store where
// the four are in range; the arrays start 16-byte aligned).
__global__ void __launch_bounds__(NTO) k_open_offsets(const int* __restrict__ t_cnt, int T,
                                                      int* __restrict__ t_off, int* count) {
  constexpr int NWP = NTO / 32;
  __shared__ int s_scr[NWP + 1];
  int carry = 0;
  for (int c0 = 0; c0 < T; c0 += 4 * NTO) {
    const int i0 = c0 + 4 * threadIdx.x;
    int v[4];
    if (i0 + 3 < T) {
      const int4 q = *reinterpret_cast<const int4*>(t_cnt + i0);
      v[0] = q.x;
      v[1] = q.y;
      v[2] = q.z;
      v[3] = q.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = i0 + j < T ? t_cnt[i0 + j] : 0;
    }
    int tot;
    const int run = carry + block_excl_scan<NWP>(v[0] + v[1] + v[2] + v[3], 0, OpAdd(), s_scr, &tot);
    const int o[4] = {run, run + v[0], run + v[0] + v[1], run + v[0] + v[1] + v[2]};
    if (i0 + 3 < T) {
      *reinterpret_cast<int4*>(t_off + i0) = make_int4(o[0], o[1], o[2], o[3]);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (i0 + j < T) t_off[i0 + j] = o[j];
    }
    carry += tot;
  }
  if (threadIdx.x == 0) *count = carry;
}

// Per round of vectors: block scan of the threads' counts, positions
// collected in shared memory in stream order, one coalesced copy out.
__global__ void __launch_bounds__(ONT) k_open_scatter(const uint8_t* __restrict__ kind, int n,
                                                      const int* __restrict__ t_off,
                                                      int* __restrict__ pos, int64_t cap) {
  __shared__ int s_pos[OROUND];
  __shared__ int s_scr[ONW + 1];
  const int t = blockIdx.x, tid = threadIdx.x;
  const int e0 = t * OTILE + tid * 16;
  unsigned m[OVEC];
#pragma unroll
  for (int r = 0; r < OVEC; ++r) {
    bool bad;  // bytes above 3 were reported by k_open_count
    m[r] = vec_open_mask(kind, n, e0 + r * OROUND, &bad);
  }
  int64_t off = t_off[t];
#pragma unroll
  for (int r = 0; r < OVEC; ++r) {
    int tot;
    int o = block_excl_scan<ONW>(popc(m[r]), 0, OpAdd(), s_scr, &tot);
    for (unsigned mm = m[r]; mm; mm &= mm - 1) s_pos[o++] = e0 + r * OROUND + lowest_set(mm);
    __syncthreads();
    for (int k = tid; k < tot; k += ONT)
      if (off + k < cap) pos[off + k] = s_pos[k];
    off += tot;
    __syncthreads();  // s_pos is refilled by the next round
  }
}

}  // namespace tb

#endif  // TB_OPEN_KERNELS_CUH
