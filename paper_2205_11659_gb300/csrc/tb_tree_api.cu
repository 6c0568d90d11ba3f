// tb_tree_api.cu -- the tree scans of include/tb.h: argument checks and the
// C entry points over the launch sequences of tb_tree_launch.cuh.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "tb.h"
#include "tb_internal.h"

#define TB_PHASE_MARK(stream) tb_internal::phase_mark(stream)
#define TB_WITHHELD_TILE() tb_internal::withheld_tile()
#include "tb_tree_launch.cuh"

using namespace tb;
using namespace tb::launch;

namespace tb_internal {
size_t tree_ws_bytes(int op, int64_t n) {
  if (n <= 0 || n > kMaxN) return 0;
  return tree_layout(n, op == TB_OP_TREE_BACKWARD).total;
}
}  // namespace tb_internal

extern "C" {

tb_status tb_tree_scan(int monoid, int dir, const uint8_t* kind, int64_t n, int64_t num_joints,
                       const void* in, void* out, void* ws, size_t ws_bytes, int32_t* d_status,
                       void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tb_internal::phase_reset();
  if (monoid < TB_MONOID_BBOX_ISECT || monoid > TB_MONOID_RIGID_F32) return TB_ERR_INVALID_ARG;
  if (dir != TB_DOWN && dir != TB_UP) return TB_ERR_INVALID_ARG;
  tb_status st = check_common(kind, n, num_joints, ws, d_status);
  if (st != TB_OK) return st;
  if (num_joints > 0) {
    if (in == nullptr || out == nullptr || !aligned(in, 16) || !aligned(out, 16) || in == out)
      return TB_ERR_INVALID_ARG;
  }
  const TreeLayout L = tree_layout(n, false);
  if (n > 0 && ws_bytes < L.total) return TB_ERR_WORKSPACE;
  if (n == 0) return cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) == cudaSuccess ? TB_OK : TB_ERR_CUDA;
  TreeWs w;
  st = prelude(kind, n, (int)num_joints, L, ws, d_status, s, &w);
  if (st != TB_OK || num_joints == 0) {
    if (st == TB_OK) TB_PHASE_MARK(s);
    return st;
  }
  switch (monoid) {
    case TB_MONOID_BBOX_ISECT:
      st = scan_dir<MonoidIsect>(dir, w, in, out, d_status, s);
      break;
    case TB_MONOID_BBOX_UNION:
      st = scan_dir<MonoidUnion>(dir, w, in, out, d_status, s);
      break;
    case TB_MONOID_ADD_I32:
      st = scan_dir<MonoidAddI32>(dir, w, in, out, d_status, s);
      break;
    case TB_MONOID_RIGID_F32:
      st = scan_dir<MonoidRigid>(dir, w, in, out, d_status, s);
      break;
    default:
      st = scan_dir<MonoidAffine>(dir, w, in, out, d_status, s);
      break;
  }
  if (st == TB_OK) TB_PHASE_MARK(s);
  return st;
}

tb_status tb_tree_scan_affine_backward(const uint8_t* kind, int64_t n, int64_t num_joints,
                                       const float* local, const float* grad_world,
                                       float* grad_local, void* ws, size_t ws_bytes,
                                       int32_t* d_status, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tb_internal::phase_reset();
  tb_status st = check_common(kind, n, num_joints, ws, d_status);
  if (st != TB_OK) return st;
  if (num_joints > 0) {
    if (local == nullptr || grad_world == nullptr || grad_local == nullptr || !aligned(local, 16) ||
        !aligned(grad_world, 16) || !aligned(grad_local, 16) || grad_local == local ||
        grad_local == grad_world)
      return TB_ERR_INVALID_ARG;
  }
  const TreeLayout L = tree_layout(n, true);
  if (n > 0 && ws_bytes < L.total) return TB_ERR_WORKSPACE;
  if (n == 0) return cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) == cudaSuccess ? TB_OK : TB_ERR_CUDA;
  TreeWs w;
  st = prelude(kind, n, (int)num_joints, L, ws, d_status, s, &w);
  if (st != TB_OK || num_joints == 0) {
    if (st == TB_OK) TB_PHASE_MARK(s);
    return st;
  }
  unsigned char* b = static_cast<unsigned char*>(ws);
  void* world = b + L.world;
  void* acc = b + L.acc;
  st = launch_jstruct<MonoidAffine, true>(w, local, s);
  if (st != TB_OK) return st;
  st = launch_adjoint(w, local, grad_world, world, acc, grad_local, d_status, s);
  if (st != TB_OK) return st;
  TB_PHASE_MARK(s);
  return TB_OK;
}

tb_status tb_tree_scan_affine_backward_reuse(const uint8_t* kind, int64_t n, int64_t num_joints,
                                             const float* local, const float* grad_world,
                                             float* grad_local, void* ws, size_t ws_bytes,
                                             int32_t* d_status, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tb_internal::phase_reset();
  tb_status st = check_common(kind, n, num_joints, ws, d_status);
  if (st != TB_OK) return st;
  if (num_joints > 0) {
    if (local == nullptr || grad_world == nullptr || grad_local == nullptr || !aligned(local, 16) ||
        !aligned(grad_world, 16) || !aligned(grad_local, 16) || grad_local == local ||
        grad_local == grad_world)
      return TB_ERR_INVALID_ARG;
  }
  const TreeLayout L = tree_layout(n, true);
  if (n > 0 && ws_bytes < L.total) return TB_ERR_WORKSPACE;
  if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess) return TB_ERR_CUDA;
  if (n == 0 || num_joints == 0) return TB_OK;
  unsigned char* b = static_cast<unsigned char*>(ws);
  TreeWs w = tree_ws(L, ws, n, (int)num_joints);
  w.status = d_status;
  // only the subtree-list counter restarts; the structure and its header stay
  if (cudaMemsetAsync(b + L.xcount, 0, 4, s) != cudaSuccess) return TB_ERR_CUDA;
  void* world = b + L.world;
  void* acc = b + L.acc;
  TB_PHASE_MARK(s);
  k_jchain<MonoidAffine><<<w.TJ, JNT, 0, s>>>(w, local, d_status);
  if (cudaGetLastError() != cudaSuccess) return TB_ERR_CUDA;
  st = launch_adjoint(w, local, grad_world, world, acc, grad_local, d_status, s);
  if (st != TB_OK) return st;
  TB_PHASE_MARK(s);
  return TB_OK;
}

tb_status tb_tree_structure(const uint8_t* kind, int64_t n, int64_t num_joints, int32_t* depth_out,
                            int32_t* parent_out, int32_t* left_sibling_out, void* ws, size_t ws_bytes,
                            int32_t* d_status, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tb_internal::phase_reset();
  tb_status st = check_common(kind, n, num_joints, ws, d_status);
  if (st != TB_OK) return st;
  if ((depth_out != nullptr && !aligned(depth_out, 4)) || (parent_out != nullptr && !aligned(parent_out, 4)) ||
      (left_sibling_out != nullptr && !aligned(left_sibling_out, 4)))
    return TB_ERR_INVALID_ARG;
  const TreeLayout L = tree_layout(n, false);
  if (n > 0 && ws_bytes < L.total) return TB_ERR_WORKSPACE;
  if (n == 0) return cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) == cudaSuccess ? TB_OK : TB_ERR_CUDA;
  TreeWs w;
  st = prelude(kind, n, (int)num_joints, L, ws, d_status, s, &w);
  if (st != TB_OK || num_joints == 0) return st;
  st = launch_jstruct<MonoidAddI32, false>(w, nullptr, s);
  if (st != TB_OK) return st;
  const size_t bytes = (size_t)num_joints * sizeof(int32_t);
  if (depth_out != nullptr &&
      cudaMemcpyAsync(depth_out, w.jdepth, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return TB_ERR_CUDA;
  if (parent_out != nullptr &&
      cudaMemcpyAsync(parent_out, w.jparent, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return TB_ERR_CUDA;
  if (left_sibling_out != nullptr) {
    if (cudaMemsetAsync(left_sibling_out, 0xff, bytes, s) != cudaSuccess) return TB_ERR_CUDA;  // -1
    TB_PHASE_MARK(s);
    k_left_sibling<<<grid_for(w.J, 256), 256, 0, s>>>(w, left_sibling_out);
    if (cudaGetLastError() != cudaSuccess) return TB_ERR_CUDA;
  }
  TB_PHASE_MARK(s);
  return TB_OK;
}

}  // extern "C"
