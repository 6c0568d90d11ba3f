// tb_open_api.cu -- tb_open_positions of include/tb.h: argument checks, the
// scratch layout (tile counts, tile offsets) and the three launches.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "tb.h"
#include "tb_internal.h"
#include "tb_open_kernels.cuh"

namespace {

using namespace tb;

constexpr int64_t kMaxN = (int64_t)INT_MAX - OTILE;

constexpr size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

int tiles(int64_t n) { return (int)((n + OTILE - 1) / OTILE); }

}  // namespace

namespace tb_internal {
size_t open_ws_bytes(int64_t n) {
  if (n <= 0 || n > kMaxN) return 0;
  return 2 * align_up((size_t)tiles(n) * 4);
}
}  // namespace tb_internal

extern "C" tb_status tb_open_positions(const uint8_t* kind, int64_t n, int32_t* pos,
                                       int64_t max_opens, int32_t* d_count, void* ws,
                                       size_t ws_bytes, int32_t* d_status, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n < 0 || n > kMaxN || max_opens < 0 || d_status == nullptr || d_count == nullptr)
    return TB_ERR_INVALID_ARG;
  if (!aligned(d_status, 4) || !aligned(d_count, 4)) return TB_ERR_INVALID_ARG;
  if (n > 0 && (kind == nullptr || ws == nullptr || !aligned(kind, 16) || !aligned(ws, 16)))
    return TB_ERR_INVALID_ARG;
  if (max_opens > 0 && (pos == nullptr || !aligned(pos, 4))) return TB_ERR_INVALID_ARG;
  if (n > 0 && ws_bytes < tb_internal::open_ws_bytes(n)) return TB_ERR_WORKSPACE;
  tb_internal::phase_reset();
  if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess) return TB_ERR_CUDA;
  if (n == 0)
    return cudaMemsetAsync(d_count, 0, sizeof(int32_t), s) == cudaSuccess ? TB_OK : TB_ERR_CUDA;
  const int T = tiles(n);
  int* t_cnt = static_cast<int*>(ws);
  int* t_off = reinterpret_cast<int*>(static_cast<unsigned char*>(ws) + align_up((size_t)T * 4));
  tb_internal::phase_mark(s);
  k_open_count<<<T, ONT, 0, s>>>(kind, (int)n, t_cnt, d_status);
  tb_internal::phase_mark(s);
  k_open_offsets<<<1, NTO, 0, s>>>(t_cnt, T, t_off, d_count);
  tb_internal::phase_mark(s);
  k_open_scatter<<<T, ONT, 0, s>>>(kind, (int)n, t_off, pos, max_opens);
  if (cudaGetLastError() != cudaSuccess) return TB_ERR_CUDA;
  tb_internal::phase_mark(s);
  return TB_OK;
}
