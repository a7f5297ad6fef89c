// k1d_wide.cu -- the second tier of the float32 1-D kernel: launch of its
// wide form (k1d.cuh) over the chunks the first launch listed.
#include "k1d.cuh"
#include "devonce.h"
#include "launch.h"

namespace swc {

namespace {
constexpr int kM1 = 63;  // as k1d.cu
}

template <bool UNIT>
static cudaError_t launch_wide(const K1DParams& p, int grid, int warps, size_t smem, cudaStream_t st) {
  static std::atomic<uint64_t> attr_done{0};  // one bit per device
  cudaError_t e = once_per_device(attr_done, [] {
    return cudaFuncSetAttribute(k1d_kernel<kM1, true, UNIT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                220 * 1024);
  });
  if (e != cudaSuccess) return e;
  k1d_kernel<kM1, true, UNIT, true><<<grid, 32 * warps, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t k1d_wide_launch(const K1DParams& p, int grid, int warps, size_t smem, cudaStream_t st) {
  return p.stride == 1 ? launch_wide<true>(p, grid, warps, smem, st) : launch_wide<false>(p, grid, warps, smem, st);
}

}  // namespace swc
