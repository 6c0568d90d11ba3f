/* tb_monoid.cuh -- tree scans over a monoid of the caller's own, compiled
 * into the caller's translation unit (header-only; CUDA C++ for sm_103a).
 *
 * The library's tb_tree_scan (tb.h) covers four built-in monoids.  The
 * paper's scans work for any associative operation with an identity (Sec. 1
 * and Sec. 13; neither commutativity nor idempotence is needed).  For
 * another one, describe it as a type
 *
 *   struct MyMonoid {
 *     using V = ...;                                   // trivially copyable,
 *                                                      // a multiple of 4 bytes,
 *                                                      // at most 48 bytes
 *     __device__ static V identity();
 *     __device__ static V combine(const V& a, const V& b);  // a is earlier
 *     __device__ static V load(const void* p, int64_t i);   // value i of p
 *     __device__ static void store(void* p, int64_t i, const V& v);
 *   };
 *
 * and call tb::tree_scan<MyMonoid>(dir, kind, n, num_joints, in, out, ws,
 * ws_bytes, d_status, stream) from host code compiled by nvcc.  Arguments,
 * layout, ownership, the meaning of TB_DOWN / TB_UP and the error behaviour
 * are those of tb_tree_scan; ws needs tb::tree_scan_workspace_size(n) bytes
 * and in / out 16-byte alignment.  The kernels are instantiated in the
 * caller's code, not taken from the library, and do not record the
 * library's tracing events. */
#ifndef TB_MONOID_CUH
#define TB_MONOID_CUH

#include "tb.h"
#include "../paper_2205_11659_gb300/csrc/tb_tree_launch.cuh"

namespace tb {
// Internal linkage, like the launch sequence it calls: each shared object
// that includes this header keeps its own kernels and launch state.
namespace {

inline size_t tree_scan_workspace_size(int64_t n) {
  if (n <= 0 || n > launch::kMaxN) return 0;
  return launch::tree_layout(n, false).total;
}

template <class M>
tb_status tree_scan(int dir, const uint8_t* kind, int64_t n, int64_t num_joints, const void* in,
                    void* out, void* ws, size_t ws_bytes, int32_t* d_status, cudaStream_t stream) {
  static_assert(sizeof(typename M::V) <= launch::kValBytes,
                "a monoid value may take at most 48 bytes of workspace per joint");
  static_assert(sizeof(typename M::V) % 4 == 0,
                "a monoid value is whole 32-bit words (warp shuffles move it word by word)");
  if (dir != TB_DOWN && dir != TB_UP) return TB_ERR_INVALID_ARG;
  tb_status st = launch::check_common(kind, n, num_joints, ws, d_status);
  if (st != TB_OK) return st;
  if (num_joints > 0 && (in == nullptr || out == nullptr || !launch::aligned(in, 16) ||
                         !launch::aligned(out, 16) || in == out))
    return TB_ERR_INVALID_ARG;
  const launch::TreeLayout L = launch::tree_layout(n, false);
  if (n > 0 && ws_bytes < L.total) return TB_ERR_WORKSPACE;
  if (n == 0)
    return cudaMemsetAsync(d_status, 0, sizeof(int32_t), stream) == cudaSuccess ? TB_OK : TB_ERR_CUDA;
  TreeWs w;
  st = launch::prelude(kind, n, (int)num_joints, L, ws, d_status, stream, &w);
  if (st != TB_OK || num_joints == 0) return st;
  return launch::scan_dir<M>(dir, w, in, out, d_status, stream);
}

}  // namespace
}  // namespace tb

#endif  // TB_MONOID_CUH
