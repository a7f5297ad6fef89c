// common.cuh -- device helpers shared by the swcorr kernels (sm_103a).
//
// Inline PTX for mbarriers and TMA (cp.async.bulk.tensor), bounded waits
// that latch an error instead of hanging, and the status block layout.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kparams.h"

namespace swc {

// ~1 s at 2 GHz: a TMA that has not landed by then is not coming.
constexpr long long WAIT_LIMIT_CYCLES = 2000000000ll;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase.  Returns false (and latches
// ERRBIT_TIMEOUT) if the phase did not complete within WAIT_LIMIT_CYCLES.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t* status) {
  if (mbar_try_wait(bar, parity)) return true;
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > WAIT_LIMIT_CYCLES) {
      if (status) atomicOr(status + ST_ERROR, ERRBIT_TIMEOUT);
      return false;
    }
  }
  return true;
}

// 2-D tiled TMA load: box at coordinates (x = innermost, y) into smem,
// completing `bytes` on the mbarrier.  x * element size must be a multiple of
// 16 bytes (the caller guarantees it); y may be negative or past the end
// (zero fill).
__device__ __forceinline__ void tma_load_2d(void* smem_dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* smem_dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// int64 -> float32 through two 32-bit halves, v = hi * 2^32 + lo with lo the
// low word read as signed (so lo in [-2^31, 2^31) and hi = round-half-up of
// v / 2^32). For |v| < 2^31, hi = 0 and the result is v correctly rounded;
// above that |v| >= 2^31 and the three roundings (hi when |hi| > 2^24, lo,
// the fma) keep the relative error below 2^-22. Two 32-bit conversions and
// an fma issue faster than one 64-bit conversion.
__device__ __forceinline__ float i64_to_f32(long long v) {
  const int lo = (int)(unsigned)(unsigned long long)v;
  const int hi = (int)(v >> 32) + (int)((unsigned)lo >> 31);
  return fmaf((float)hi, 4294967296.0f, (float)lo);
}

// Clamp to [-1, 1] that keeps NaN, in one instruction: min of |v| and 1
// with the sign of v (sign(v) xor sign(1)); .NaN propagates a NaN input.
__device__ __forceinline__ float clamp1_nan(float v) {
  float r;
  asm("min.NaN.xorsign.abs.f32 %0, %1, 0f3F800000;" : "=f"(r) : "f"(v));
  return r;
}

__device__ __forceinline__ uint4 lds128(const void* p) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(smem_u32(p)));
  return v;
}

__device__ __forceinline__ void stg128(float* p, float a, float b, float c, float d) {
  asm volatile("st.global.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

}  // namespace swc
