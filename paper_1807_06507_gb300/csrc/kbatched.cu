// kbatched.cu -- one persistent launch over the tiles of many 2-D uint16
// scenes of uneven sizes and window sizes.
//
// Work items (scene, column strip, row block) sit in a device array ordered
// largest cost first; each CTA (one warp) takes the next item from an atomic
// counter and runs the fused 2-D kernel body specialised for that scene's
// window width.  The counter is reset by a memset node in front of the
// kernel node of the CUDA graph the plan replays on every run.
#include "k2d_u16.cuh"
#include "launch.h"

namespace swc {

template <int KW, bool WIDE>
__device__ __forceinline__ bool run_item(const Scene2D& sc, int strip, int rb, const Ring2D& rg, uint32_t& seq,
                                         uint32_t* status) {
  return process_item_2d_u16<8, KW, true, WIDE>(sc, strip, rb, rg, seq, status);
}

__global__ void __launch_bounds__(32) kbatched_kernel(const __grid_constant__ KBatchParams p) {
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
    // 32-bit engine for small windows (kw <= 9, kh*kw <= 64), 64-bit otherwise
    const int key = sc.wide ? 100 + sc.kw : sc.kw;
    switch (key) {
#define X(KW)                                                           \
  case KW:                                                              \
    ok = run_item<KW, false>(sc, it.strip, it.rb, rg, seq, p.status);  \
    break;
#define XW(KW)                                                          \
  case 100 + KW:                                                        \
    ok = run_item<KW, true>(sc, it.strip, it.rb, rg, seq, p.status);   \
    break;
      X(1) X(3) X(5) X(7) X(9)
      XW(1) XW(3) XW(5) XW(7) XW(9) XW(11) XW(13) XW(15) XW(17) XW(19) XW(21) XW(23) XW(25) XW(27) XW(29) XW(31)
#undef X
#undef XW
      default:
        if (lane == 0) atomicOr(p.status + ST_ERROR, ERRBIT_BAD_ARG);
        ok = false;
    }
    if (!ok) return;
  }
}

int kbatched_ring_row() { return Geo2D<8, 31>::RWS; }

const void* kbatched_kernel_ptr() { return reinterpret_cast<const void*>(kbatched_kernel); }

cudaError_t kbatched_prepare() {
  return cudaFuncSetAttribute(kbatched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

cudaError_t kbatched_launch(const KBatchParams& p, int grid, size_t smem, cudaStream_t st) {
  kbatched_kernel<<<grid, 32, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace swc
