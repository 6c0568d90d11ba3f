// tb_device_once.h -- host-side launch settings that are made once per
// device: a kernel's raised dynamic shared-memory limit, the device's SM
// count.  A CUDA function attribute belongs to the current device's copy of
// the kernel, so a flag kept per process would skip the setting on the
// second device a process uses, and that device's launch would fail.
//
// Internal linkage (an unnamed namespace), like the launch sequences that
// use it: each shared object keeps its own flags.  Devices 0..63 get one bit
// each in a 64-bit atomic mask; a setting for a higher ordinal is simply made
// on every call.  Two host threads that race on a device's first call may
// both make the setting, which is harmless: it is idempotent.
#ifndef TB_DEVICE_ONCE_H
#define TB_DEVICE_ONCE_H

#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>

namespace tb {
namespace {

constexpr int kOnceDevices = 64;

template <class Set>
inline cudaError_t once_per_device(std::atomic<unsigned long long>& done, Set set) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool tracked = dev >= 0 && dev < kOnceDevices;
  const unsigned long long bit = tracked ? 1ull << dev : 0ull;
  if (tracked && (done.load(std::memory_order_acquire) & bit) != 0) return cudaSuccess;
  e = set();
  if (e == cudaSuccess && tracked) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// Raises `kernel`'s dynamic shared-memory limit to `bytes` on the current
// device, the first time this call site runs on that device.
template <class K>
inline cudaError_t smem_limit_once(std::atomic<unsigned long long>& done, K kernel, size_t bytes) {
  return once_per_device(done, [&] {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  });
}

// Number of SMs of the current device (looked up once per device); 0 when
// the query fails.
inline int current_device_sms() {
  static std::atomic<int> cached[kOnceDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  const bool tracked = dev >= 0 && dev < kOnceDevices;
  if (tracked) {
    const int c = cached[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (tracked && sms > 0) cached[dev].store(sms, std::memory_order_relaxed);
  return sms;
}

}  // namespace
}  // namespace tb

#endif  // TB_DEVICE_ONCE_H
