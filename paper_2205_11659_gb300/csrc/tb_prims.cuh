// tb_prims.cuh -- the few hardware primitives the kernels use: warp
// shuffles and votes, acquire/release accesses for the cross-block
// look-back, bounded-wait backoff, atomics and read-only 128-bit loads.
#ifndef TB_PRIMS_CUH
#define TB_PRIMS_CUH

#include <cstdint>

// Dynamic shared memory of a kernel, 128-byte aligned.
#define TB_DYNAMIC_SMEM(name) extern __shared__ __align__(128) unsigned char name[]

namespace tb {

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }

__device__ __forceinline__ int shfl_up(int v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ int shfl_down(int v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ int shfl_idx(int v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ float shfl_up(float v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ float shfl_down(float v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ int shfl_xor(int v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ float shfl_xor(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ unsigned ballot(bool p) { return __ballot_sync(0xffffffffu, p); }
__device__ __forceinline__ int popc(unsigned x) { return __popc(x); }
__device__ __forceinline__ int lowest_set(unsigned x) { return __ffs(x) - 1; }  // -1 if none
__device__ __forceinline__ bool block_or(bool p) { return __syncthreads_or(p) != 0; }

// Acquire load / release store at GPU scope: a block that observes another
// block's published flag also observes everything written before it.
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire_i32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_i32(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Backoff between polls of a flag another block will set.
__device__ __forceinline__ void poll_backoff(unsigned it) {
  if (it > 16) __nanosleep(it > 1024 ? 1000 : 64);
}

__device__ __forceinline__ unsigned atomic_add_u32(unsigned* p, unsigned v) { return atomicAdd(p, v); }
__device__ __forceinline__ int atomic_cas_i32(int* p, int cmp, int v) { return atomicCAS(p, cmp, v); }
__device__ __forceinline__ void atomic_min_i32(int* p, int v) { atomicMin(p, v); }

// 16-byte asynchronous global -> shared copy (cp.async.cg, bypassing L1),
// committed as one group and awaited with cp_async_wait_all.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// 128-bit read-only loads of input streams (ld.global.nc.v4).
__device__ __forceinline__ uint4 ld_nc_u4(const void* p) { return __ldg(reinterpret_cast<const uint4*>(p)); }
__device__ __forceinline__ uint2 ld_nc_u2(const void* p) { return __ldg(reinterpret_cast<const uint2*>(p)); }
__device__ __forceinline__ float4 ld_nc_f4(const void* p) { return __ldg(reinterpret_cast<const float4*>(p)); }

}  // namespace tb

#endif  // TB_PRIMS_CUH
