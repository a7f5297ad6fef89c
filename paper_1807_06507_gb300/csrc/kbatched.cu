// kbatched.cu -- one persistent launch over the tiles of many 2-D uint16
// scenes of uneven sizes and window sizes.
//
// Work items (scene, column strip, row block) sit in device arrays ordered
// largest cost first, one array per class of kernel body (32-bit sums for
// windows of at most 64 cells and 9 columns; 64-bit up to 17 columns; 64-bit
// above), so that each launch keeps the occupancy its bodies allow; each CTA
// (one warp) takes the next item from its array's atomic counter and runs
// the fused 2-D kernel body specialised for that scene's window width.  The
// plan replays one CUDA graph: a memset node resetting the counters, then
// one kernel node per non-empty class.
#include "k2d_u16.cuh"
#include "launch.h"

namespace swc {

template <int KW, bool WIDE>
__device__ __forceinline__ bool run_item(const Scene2D& sc, int strip, int rb, const Ring2D& rg, uint32_t& seq,
                                         uint32_t* status) {
  return process_item_2d_u16<8, KW, true, WIDE>(sc, strip, rb, rg, seq, status);
}

// One instance per class of body: 0 = 32-bit engine (windows of at most 64
// cells and 9 columns, 16 resident CTAs per SM), 1 = 64-bit engine up to 17
// columns (12 per SM), 2 = 64-bit engine above (8 per SM).
template <int CLS>
__global__ void __launch_bounds__(32, CLS == 0 ? 16 : (CLS == 1 ? 12 : 8)) kbatched_kernel(
    const __grid_constant__ KBatchParams p) {
  constexpr bool WIDE = CLS != 0;
  constexpr int RWS = Geo2D<8, 31>::RWS;  // the same for every instance with M = 8
  static_assert(Geo2D<8, 3>::RWS == RWS && Geo2D<8, 17>::RWS == RWS, "ring rows differ between instances");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Ring2D rg;
  rg.NR = p.NR;
  rg.PF = p.PF;
  rg.rx = reinterpret_cast<uint16_t*>(smem_raw);
  rg.ry = rg.rx + (size_t)p.NR * RWS;
  rg.lx = rg.ry + (size_t)p.NR * RWS;
  rg.ly = rg.lx + (size_t)p.NR * RWS;
  rg.bar = reinterpret_cast<uint64_t*>(rg.ly + (size_t)p.NR * RWS);
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
    switch (sc.kw) {
#define X(KW)                                                         \
  case KW:                                                            \
    if constexpr (CLS < 2) ok = run_item<KW, WIDE>(sc, it.strip, it.rb, rg, seq, p.status); \
    break;
      X(1) X(3) X(5) X(7) X(9)
#undef X
#define X(KW)                                                         \
  case KW:                                                            \
    if constexpr (CLS == 1) ok = run_item<KW, true>(sc, it.strip, it.rb, rg, seq, p.status); \
    break;
      X(11) X(13) X(15) X(17)
#undef X
#define X(KW)                                                         \
  case KW:                                                            \
    if constexpr (CLS == 2) ok = run_item<KW, true>(sc, it.strip, it.rb, rg, seq, p.status); \
    break;
      X(19) X(21) X(23) X(25) X(27) X(29) X(31)
#undef X
      default:
        if (lane == 0) atomicOr(p.status + ST_ERROR, ERRBIT_BAD_ARG);
        ok = false;
    }
    if (!ok) return;
  }
}

int kbatched_ring_row() { return Geo2D<8, 31>::RWS; }

const void* kbatched_kernel_ptr(int cls) {
  return cls == 0 ? reinterpret_cast<const void*>(kbatched_kernel<0>)
                  : cls == 1 ? reinterpret_cast<const void*>(kbatched_kernel<1>)
                             : reinterpret_cast<const void*>(kbatched_kernel<2>);
}

cudaError_t kbatched_prepare() {
  cudaError_t e = cudaFuncSetAttribute(kbatched_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kbatched_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kbatched_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  return e;
}

cudaError_t kbatched_launch(const KBatchParams& p, int cls, int grid, size_t smem, cudaStream_t st) {
  if (cls == 0)
    kbatched_kernel<0><<<grid, 32, smem, st>>>(p);
  else if (cls == 1)
    kbatched_kernel<1><<<grid, 32, smem, st>>>(p);
  else
    kbatched_kernel<2><<<grid, 32, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace swc
