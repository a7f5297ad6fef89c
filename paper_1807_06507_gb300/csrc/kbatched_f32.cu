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

namespace {

constexpr int kRWS = Geo2DF<8, 31>::RWS;  // the same for every instance with M = 8
static_assert(Geo2DF<8, 1>::RWS == kRWS && Geo2DF<8, 17>::RWS == kRWS, "ring rows differ between instances");

// One instance per window width (class (KW - 1) / 2), so that each kernel
// holds the registers of its own body only.
template <int KW>
__global__ void __launch_bounds__(32, 12) kbatched_f32_kernel(const __grid_constant__ KBatchParams p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Ring2DF rg;
  rg.NR = p.NR;
  rg.PF = p.PF;
  rg.rx = reinterpret_cast<float*>(smem_raw);
  rg.ry = rg.rx + (size_t)p.NR * kRWS;
  rg.lx = rg.ry + (size_t)p.NR * kRWS;
  rg.ly = rg.lx + (size_t)p.NR * kRWS;
  rg.bar = reinterpret_cast<uint64_t*>(rg.ly + (size_t)p.NR * kRWS);
  __shared__ uint32_t pend[kPend2D];
  __shared__ int npend;
  rg.pend = pend;
  rg.npend = &npend;
  const int lane = threadIdx.x;
  if (lane == 0) {
    for (int s = 0; s < p.NR; s++) mbar_init(rg.bar + s, 1);
    fence_mbar_init();
  }
  __syncwarp();
  uint32_t seq = 0;
  while (true) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(p.counter, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= (uint32_t)p.n_items) break;
    const BatchItem it = p.items[item];
    const Scene2D sc = p.scenes[it.scene];
    bool ok = true;
    if (sc.kw == KW) {
      ok = process_item_2d_f32<8, KW, true>(sc, it.strip, it.rb, rg, seq, p.status);
    } else {
      if (lane == 0) atomicOr(p.status + ST_ERROR, ERRBIT_BAD_ARG);
      ok = false;
    }
    if (!ok) return;
  }
}

}  // namespace

int kbatched_f32_ring_row() { return kRWS; }

#define SWC_KB32_CASES(X) X(1) X(3) X(5) X(7) X(9) X(11) X(13) X(15) X(17) X(19) X(21) X(23) X(25) X(27) X(29) X(31)

const void* kbatched_f32_kernel_ptr(int cls) {
  switch (2 * cls + 1) {
#define X(KW) \
  case KW:    \
    return reinterpret_cast<const void*>(kbatched_f32_kernel<KW>);
    SWC_KB32_CASES(X)
#undef X
    default:
      return nullptr;
  }
}

cudaError_t kbatched_f32_prepare() {
  cudaError_t e = cudaSuccess;
  for (int c = 0; c < 16 && e == cudaSuccess; c++)
    e = cudaFuncSetAttribute(kbatched_f32_kernel_ptr(c), cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  return e;
}

cudaError_t kbatched_f32_launch(const KBatchParams& p, int cls, int grid, size_t smem, cudaStream_t st) {
  switch (2 * cls + 1) {
#define X(KW)                                              \
  case KW:                                                 \
    kbatched_f32_kernel<KW><<<grid, 32, smem, st>>>(p);    \
    break;
    SWC_KB32_CASES(X)
#undef X
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace swc
