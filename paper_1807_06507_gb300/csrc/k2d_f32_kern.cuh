// k2d_f32_kern.cuh -- the fused 2-D float32 kernel's entry point and launch
// helper, instantiated by k2d_f32_p0.cu .. k2d_f32_p7.cu (eight pairs of
// window widths, compiled in parallel).
#pragma once

#include "k2d_f32.cuh"
#include "devonce.h"
#include "launch.h"

namespace swc {

#ifndef SWC_K2DF_MINB
#define SWC_K2DF_MINB 12  // resident one-warp CTAs per SM the float32 2-D kernel is compiled for
#endif
template <int M, int KW, bool TMA, int TIER>
__global__ void __launch_bounds__(32, SWC_K2DF_MINB) k2d_f32_kernel(const __grid_constant__ K2DParams p) {
  using G = Geo2DF<M, KW>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Ring2DF rg;
  rg.NR = p.NR;
  rg.PF = p.PF;
  rg.rx = reinterpret_cast<float*>(smem_raw);
  rg.ry = rg.rx + (size_t)p.NR * G::RWS;
  rg.lx = rg.ry + (size_t)p.NR * G::RWS;
  rg.ly = rg.lx + (size_t)p.NR * G::RWS;
  rg.bar = reinterpret_cast<uint64_t*>(rg.ly + (size_t)p.NR * G::RWS);
  __shared__ uint32_t pend[kPend2D];  // windows the lane re-march could not certify
  __shared__ int npend;
  rg.pend = pend;
  rg.npend = &npend;
  if (threadIdx.x == 0) {
    for (int s = 0; s < p.NR; s++) mbar_init(rg.bar + s, 1);
    fence_mbar_init();
    if (TMA) {
      prefetch_tmap(&p.tmx);
      prefetch_tmap(&p.tmy);
      if (G::TAIL > 0) {
        prefetch_tmap(&p.tmx_t);
        prefetch_tmap(&p.tmy_t);
      }
    }
  }
  __syncwarp();
  Scene2D sc = p.sc;
  sc.tmx = &p.tmx;
  sc.tmy = &p.tmy;
  sc.tmx_t = &p.tmx_t;
  sc.tmy_t = &p.tmy_t;
  uint32_t seq = 0;
  // work items, or (second-tier launch) the tasks the previous launch listed
  const int n_iter = TIER == TIER_TASK ? min(*sc.redo_count, sc.redo_cap) : p.n_items;
  for (int it = blockIdx.x; it < n_iter; it += gridDim.x) {
    int strip, j0, j1, slot = 0;
    uint32_t lanes = 0u;
    if constexpr (TIER == TIER_TASK) {
      const RedoTask2D t = sc.redo_tasks[it];
      strip = t.strip;
      j0 = t.j0;
      j1 = t.j1;
      lanes = t.lanes;
      slot = t.range_slot;
    } else {
      const int rbi = it / sc.n_strips;
      strip = it - rbi * sc.n_strips;
      j0 = (p.rb0 + rbi) * sc.TJ;
      j1 = min(j0 + sc.TJ, sc.OH);
    }
    if (!process_rows_2d_f32<M, KW, TMA, TIER>(sc, strip, j0, j1, lanes, slot, rg, seq, p.status)) return;
  }
}

template <int M, int KW, bool TMA, int TIER>
static cudaError_t launch_t(const K2DParams& p, int grid, size_t smem, cudaStream_t st) {
  static std::atomic<uint64_t> attr_done{0};  // one bit per device
  cudaError_t e = once_per_device(attr_done, [] {
    return cudaFuncSetAttribute(k2d_f32_kernel<M, KW, TMA, TIER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                200 * 1024);
  });
  if (e != cudaSuccess) return e;
  k2d_f32_kernel<M, KW, TMA, TIER><<<grid, 32, smem, st>>>(p);
  return cudaGetLastError();
}

template <int KW>
static cudaError_t launch_kw(const K2DParams& p, int grid, size_t smem, cudaStream_t st, bool tma, int tier) {
  switch (tier) {
    case TIER_LIST:
      return tma ? launch_t<8, KW, true, TIER_LIST>(p, grid, smem, st) : launch_t<8, KW, false, TIER_LIST>(p, grid, smem, st);
    case TIER_TASK:
      return tma ? launch_t<8, KW, true, TIER_TASK>(p, grid, smem, st) : launch_t<8, KW, false, TIER_TASK>(p, grid, smem, st);
    default:
      return tma ? launch_t<8, KW, true, TIER_IN_PLACE>(p, grid, smem, st)
                 : launch_t<8, KW, false, TIER_IN_PLACE>(p, grid, smem, st);
  }
}

// A part's launcher: the instances for the window widths KW1 and KW2.
#define SWC_K2DF_PART(NAME, KW1, KW2)                                                                    \
  cudaError_t NAME(int kw, const K2DParams& p, int grid, size_t smem, cudaStream_t st, bool tma, int tier) { \
    switch (kw) {                                                                                     \
      case KW1: return launch_kw<KW1>(p, grid, smem, st, tma, tier);                                  \
      case KW2: return launch_kw<KW2>(p, grid, smem, st, tma, tier);                                  \
      default: return cudaErrorInvalidValue;                                                          \
    }                                                                                                 \
  }

}  // namespace swc
