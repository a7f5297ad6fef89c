// k1d.cu -- launch of the fused 1-D correlation kernel.
#include "k1d.cuh"
#include "devonce.h"
#include "launch.h"

namespace swc {

constexpr int kM1 = 63;  // outputs per lane per chunk (odd: conflict-free strided shared-memory reads)

int k1d_outputs_per_lane() { return kM1; }

template <bool F32, bool UNIT>
static cudaError_t launch(const K1DParams& p, int grid, int warps, size_t smem, cudaStream_t st) {
  static std::atomic<uint64_t> attr_done{0};  // one bit per device
  cudaError_t e = once_per_device(attr_done, [] {
    return cudaFuncSetAttribute(k1d_kernel<kM1, F32, UNIT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  });
  if (e != cudaSuccess) return e;
  k1d_kernel<kM1, F32, UNIT, false><<<grid, 32 * warps, smem, st>>>(p);
  return cudaGetLastError();
}

// Separate instances for unit stride and any stride keep each kernel's fully
// unrolled slide loop alone in the instruction cache.
cudaError_t k1d_launch(const K1DParams& p, int grid, int warps, size_t smem, cudaStream_t st) {
  if (p.stride == 1)
    return p.is_f32 ? launch<true, true>(p, grid, warps, smem, st) : launch<false, true>(p, grid, warps, smem, st);
  return p.is_f32 ? launch<true, false>(p, grid, warps, smem, st) : launch<false, false>(p, grid, warps, smem, st);
}

int k1d_blocks_per_sm(bool f32, int warps, size_t smem) {
  // the unit-stride and any-stride instances share launch bounds and layout
  int b = 0;
  cudaError_t e = f32 ? cudaFuncSetAttribute(k1d_kernel<kM1, true, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             220 * 1024)
                      : cudaFuncSetAttribute(k1d_kernel<kM1, false, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             220 * 1024);
  if (e != cudaSuccess) return 0;
  e = f32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k1d_kernel<kM1, true, true, false>, 32 * warps, smem)
          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k1d_kernel<kM1, false, true, false>, 32 * warps, smem);
  return e == cudaSuccess ? b : 0;
}

}  // namespace swc
