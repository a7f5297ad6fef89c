// k3d_wide.cu -- the second tier of the float32 3-D kernel: instantiations
// and launch of its wide form (k3d.cuh), run on the items the first launch
// listed.
#include "k3d.cuh"
#include "devonce.h"
#include "launch.h"

namespace swc {

template <int K>
static cudaError_t launch_wide_k(const K3DParams& p, int grid, size_t smem, cudaStream_t st) {
  static std::atomic<uint64_t> attr_done{0};  // one bit per device
  cudaError_t e = once_per_device(attr_done, [] {
    return cudaFuncSetAttribute(k3d_kernel<kTY3, tx3<K>(), K, K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                200 * 1024);
  });
  if (e != cudaSuccess) return e;
  k3d_kernel<kTY3, tx3<K>(), K, K, true><<<grid, K3_THREADS, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t k3d_wide_launch(int k, const K3DParams& p, int grid, size_t smem, cudaStream_t st) {
  switch (k) {
#define X(K) \
  case K:    \
    return launch_wide_k<K>(p, grid, smem, st);
    X(1) X(3) X(5) X(7) X(9) X(11) X(13) X(15)
#undef X
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace swc
