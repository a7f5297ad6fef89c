// k1d.cu -- launch of the fused 1-D correlation kernel.
#include "k1d.cuh"
#include "launch.h"

namespace swc {

constexpr int kM1 = 63;  // outputs per lane per chunk (odd: conflict-free strided shared-memory reads)

int k1d_outputs_per_lane() { return kM1; }

cudaError_t k1d_launch(const K1DParams& p, int grid, size_t smem, cudaStream_t st) {
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(k1d_kernel<kM1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  k1d_kernel<kM1><<<grid, 32, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace swc
