// kbatched_f32.cu -- one persistent launch over the tiles of many 2-D
// float32 scenes of uneven sizes and window sizes.
//
// The float32 counterpart of kbatched.cu: work items (scene, column strip,
// row block) sit in a device array ordered largest cost first; each CTA (one
// warp) takes the next item from an atomic counter and runs the fused 2-D
// float32 body (k2d_f32.cuh: per-lane fixed-point map, exact integer sums,
// per-window certificate, second-tier re-march of the lanes it leaves
// uncertified).  Scenes are grouped by window width, one kernel instance per
// width; the plan replays one CUDA graph: a memset node resetting the
// counters, then one launch per width that has scenes.
#include "k2d_f32.cuh"
#include "launch.h"

namespace swc {

int kbatched_f32_ring_row() { return Geo2DF<8, 31>::RWS; }

const void* kbatched_f32_kernel_ptr(int cls) {
  const int kw = 2 * cls + 1;
  return kw <= 15 ? kbatched_f32_kernel_ptr_p0(kw) : kbatched_f32_kernel_ptr_p1(kw);
}

cudaError_t kbatched_f32_prepare() {
  cudaError_t e = cudaSuccess;
  for (int c = 0; c < 16 && e == cudaSuccess; c++)
    e = cudaFuncSetAttribute(kbatched_f32_kernel_ptr(c), cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  return e;
}

cudaError_t kbatched_f32_launch(const KBatchParams& p, int cls, int grid, size_t smem, cudaStream_t st) {
  const int kw = 2 * cls + 1;
  if (cls < 0 || cls > 15) return cudaErrorInvalidValue;
  return kw <= 15 ? kbatched_f32_launch_p0(kw, p, grid, smem, st) : kbatched_f32_launch_p1(kw, p, grid, smem, st);
}

}  // namespace swc
