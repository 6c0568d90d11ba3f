// A monoid the library does not build in -- 2x2 matrices of 32-bit unsigned
// integers under the matrix product (associative, not commutative) -- scanned
// through the header-only template of include/tb_monoid.cuh.  Compiled by
// tests/test_user_monoid.py.
#include <cstdint>

#include "tb_monoid.cuh"

struct Mat2 {
  struct V {
    unsigned a, b, c, d;  // [[a, b], [c, d]]
  };
  __device__ static V identity() { return V{1u, 0u, 0u, 1u}; }
  __device__ static V combine(const V& x, const V& y) {
    return V{x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c,
             x.c * y.b + x.d * y.d};
  }
  __device__ static V load(const void* p, int64_t i) { return static_cast<const V*>(p)[i]; }
  __device__ static void store(void* p, int64_t i, const V& v) { static_cast<V*>(p)[i] = v; }
};

extern "C" size_t user_ws_size(int64_t n) { return tb::tree_scan_workspace_size(n); }

extern "C" int user_scan(int dir, const uint8_t* kind, int64_t n, int64_t num_joints,
                         const void* in, void* out, void* ws, size_t ws_bytes, int32_t* d_status,
                         void* stream) {
  return tb::tree_scan<Mat2>(dir, kind, n, num_joints, in, out, ws, ws_bytes, d_status,
                             static_cast<cudaStream_t>(stream));
}
