// kbatched_f32_kern.cuh -- the persistent float32 kernel of batched plans
// (see kbatched_f32.cu), instantiated by kbatched_f32_p0.cu and
// kbatched_f32_p1.cu (two groups of window widths, compiled in parallel).
#pragma once

#include "k2d_f32.cuh"
#include "launch.h"

namespace swc {

inline constexpr int kRWS_B32 = Geo2DF<8, 31>::RWS;  // the same for every instance with M = 8
static_assert(Geo2DF<8, 1>::RWS == kRWS_B32 && Geo2DF<8, 17>::RWS == kRWS_B32, "ring rows differ between instances");

// One instance per window width (class (KW - 1) / 2), so that each kernel
// holds the registers of its own body only.
template <int KW>
__global__ void __launch_bounds__(32, 12) kbatched_f32_kernel(const __grid_constant__ KBatchParams p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Ring2DF rg;
  rg.NR = p.NR;
  rg.PF = p.PF;
  rg.rx = reinterpret_cast<float*>(smem_raw);
  rg.ry = rg.rx + (size_t)p.NR * kRWS_B32;
  rg.lx = rg.ry + (size_t)p.NR * kRWS_B32;
  rg.ly = rg.lx + (size_t)p.NR * kRWS_B32;
  rg.bar = reinterpret_cast<uint64_t*>(rg.ly + (size_t)p.NR * kRWS_B32);
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


// A part's pointer and launch functions: the instances for KW1..KW8.
#define SWC_KB32_PART(SUFFIX, KW1, KW2, KW3, KW4, KW5, KW6, KW7, KW8)                                  \
  const void* kbatched_f32_kernel_ptr_##SUFFIX(int kw) {                                                \
    switch (kw) {                                                                                   \
      case KW1: return reinterpret_cast<const void*>(kbatched_f32_kernel<KW1>);                     \
      case KW2: return reinterpret_cast<const void*>(kbatched_f32_kernel<KW2>);                     \
      case KW3: return reinterpret_cast<const void*>(kbatched_f32_kernel<KW3>);                     \
      case KW4: return reinterpret_cast<const void*>(kbatched_f32_kernel<KW4>);                     \
      case KW5: return reinterpret_cast<const void*>(kbatched_f32_kernel<KW5>);                     \
      case KW6: return reinterpret_cast<const void*>(kbatched_f32_kernel<KW6>);                     \
      case KW7: return reinterpret_cast<const void*>(kbatched_f32_kernel<KW7>);                     \
      case KW8: return reinterpret_cast<const void*>(kbatched_f32_kernel<KW8>);                     \
      default: return nullptr;                                                                      \
    }                                                                                               \
  }                                                                                                 \
  cudaError_t kbatched_f32_launch_##SUFFIX(int kw, const KBatchParams& p, int grid, size_t smem, cudaStream_t st) { \
    switch (kw) {                                                                                   \
      case KW1: kbatched_f32_kernel<KW1><<<grid, 32, smem, st>>>(p); break;                         \
      case KW2: kbatched_f32_kernel<KW2><<<grid, 32, smem, st>>>(p); break;                         \
      case KW3: kbatched_f32_kernel<KW3><<<grid, 32, smem, st>>>(p); break;                         \
      case KW4: kbatched_f32_kernel<KW4><<<grid, 32, smem, st>>>(p); break;                         \
      case KW5: kbatched_f32_kernel<KW5><<<grid, 32, smem, st>>>(p); break;                         \
      case KW6: kbatched_f32_kernel<KW6><<<grid, 32, smem, st>>>(p); break;                         \
      case KW7: kbatched_f32_kernel<KW7><<<grid, 32, smem, st>>>(p); break;                         \
      case KW8: kbatched_f32_kernel<KW8><<<grid, 32, smem, st>>>(p); break;                         \
      default: return cudaErrorInvalidValue;                                                        \
    }                                                                                               \
    return cudaGetLastError();                                                                      \
  }

}  // namespace swc
