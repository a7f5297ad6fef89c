// devonce.h -- run a set-up step once per device (host code).
//
// Kernel attributes such as the dynamic shared-memory opt-in belong to the
// device that is current when they are set; a process that drives several
// GPUs must set them on each.  `done` keeps one bit per device ordinal.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

namespace swc {

template <class F>
cudaError_t once_per_device(std::atomic<uint64_t>& done, F&& step) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = step();  // idempotent: two threads racing here both set the attribute
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

}  // namespace swc
