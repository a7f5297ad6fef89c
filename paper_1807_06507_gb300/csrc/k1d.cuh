// k1d.cuh -- fused 1-D sliding-window correlation (uint16 or float32).
//
// The one-dimensional case of the optimized algorithm (Section 1: window
// sums in linear time like a rolling mean, then Eq. 2), for long windows
// (k up to 32*M1*stride) on long series.
//
// One CTA of NW warps per work item = a chunk of NW*32*M1 consecutive
// outputs; warp w owns the w-th 32*M1 of them:
//  * The chunk's input span (the windows of all its outputs) is loaded into
//    shared memory with 1-D TMA boxes issued by many threads at once; cells
//    before the start or past the end of the series read as 0.
//  * Values become exact integers: uint16 as they are (read in place);
//    float32 through a fixed-point map of the chunk (reference at the
//    midpoint of the chunk's range, power-of-two scale, |X| <= 2^qbits with
//    n 2^qbits < 2^31), converted in place four cells per access.  Cells off
//    the series become 0.
//  * Lane j of warp w owns M1 consecutive outputs.  The warp's span is cut
//    into segments of M1*stride cells, so lane j's first window starts at
//    segment j: q whole segments plus the first r cells of the next
//    (k = q*M1*stride + r).  Each lane sums its two segments (five streams,
//    plus the sum of the first r cells); a warp scan of the segment totals
//    gives every lane its first window as a prefix difference.  All sums are
//    modular integers (uint32 / uint64), hence exact.
//  * The lane then slides: window t+1 = window t + the stride cells that
//    enter - the stride cells that leave (products as differences:
//    x_i^2 - x_o^2 = (x_i - x_o)(x_i + x_o)), and evaluates Eq. 2 exactly in
//    int64 for each output (NaN for a zero variance).  The lane's results
//    stay in registers until the whole CTA is done with the span, which then
//    stages them for coalesced stores.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "kparams.h"
#include "k1d_params.h"

namespace swc {

__device__ __forceinline__ void tma_load_1d(void* smem_dst, const CUtensorMap* map, int x, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.1d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2}], [%3];" ::"r"(smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ float warp_min(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

struct Sums5 {
  uint32_t x, y;
  uint64_t xx, yy, xy;
  __device__ __forceinline__ void zero() { x = y = 0u; xx = yy = xy = 0ull; }
  __device__ __forceinline__ void add(int X, int Y) {
    x += (uint32_t)X;
    y += (uint32_t)Y;
    xx += (uint64_t)((long long)X * X);
    yy += (uint64_t)((long long)Y * Y);
    xy += (uint64_t)((long long)X * Y);
  }
  // window += (Xi, Yi) - (Xo, Yo)
  __device__ __forceinline__ void slide(int Xi, int Yi, int Xo, int Yo) {
    const int dx = Xi - Xo, dy = Yi - Yo;
    x += (uint32_t)dx;
    y += (uint32_t)dy;
    xx += (uint64_t)((long long)dx * (Xi + Xo));
    yy += (uint64_t)((long long)dy * (Yi + Yo));
    xy += (uint64_t)((long long)dx * Yi + (long long)Xo * dy);
  }
  __device__ __forceinline__ void add(const Sums5& o) { x += o.x; y += o.y; xx += o.xx; yy += o.yy; xy += o.xy; }
  __device__ __forceinline__ void sub(const Sums5& o) { x -= o.x; y -= o.y; xx -= o.xx; yy -= o.yy; xy -= o.xy; }
  __device__ __forceinline__ Sums5 shfl(int src) const {
    Sums5 r;
    r.x = __shfl_sync(0xffffffffu, x, src);
    r.y = __shfl_sync(0xffffffffu, y, src);
    r.xx = __shfl_sync(0xffffffffu, xx, src);
    r.yy = __shfl_sync(0xffffffffu, yy, src);
    r.xy = __shfl_sync(0xffffffffu, xy, src);
    return r;
  }
};

// Eq. 2 from exact modular window sums (the results fit in int64; the first
// moments are below 2^31 in magnitude).
__device__ __forceinline__ float pearson_exact(const Sums5& s, uint32_t n) {
  const long long sx = (int)s.x, sy = (int)s.y;
  const long long vx = (long long)((uint64_t)n * s.xx - (uint64_t)(sx * sx));
  const long long vy = (long long)((uint64_t)n * s.yy - (uint64_t)(sy * sy));
  const long long num = (long long)((uint64_t)n * s.xy - (uint64_t)(sx * sy));
  // a zero variance makes num exactly 0, so 0 * rsqrt(0) = NaN
  return clamp1_nan(i64_to_f32(num) * rsqrtf(i64_to_f32(vx) * i64_to_f32(vy)));
}

// Fixed-point map of a float32 chunk: m = midpoint of [lo, hi], scale 2^e
// with |x - m| 2^e <= 2^qbits.
__device__ __forceinline__ void fixed_point(float lo, float hi, int qbits, float& m, float& s) {
  if (!(lo <= hi)) lo = hi = 0.0f;  // a chunk with no cell on the series
  m = lo + 0.5f * (hi - lo);
  const float A = fmaxf(hi - m, m - lo);
  int e = 0;
  if (A > 0.0f) {
    int ea;
    frexpf(A, &ea);  // A < 2^ea
    e = min(max(qbits - ea, -126), 126);
  }
  s = __int_as_float((127 + e) << 23);
}

// Round to nearest of (v - m) * s (|result| <= 2^22) through the float32
// significand: adding 1.5 * 2^23 puts the integer in the low mantissa bits.
__device__ __forceinline__ int to_fixed(float v, float m, float s) {
  return __float_as_int(fmaf(v - m, s, 12582912.0f)) - 0x4B400000;
}

template <int M1, bool F32, bool UNIT>
__global__ void __launch_bounds__(128, 3) k1d_kernel(const __grid_constant__ K1DParams p) {
  constexpr int LW = 32 * M1;  // outputs per warp
  static_assert(LW % 4 == 0, "vector stores of the staged outputs");
  using T = typename std::conditional<F32, float, uint16_t>::type;
  using I = typename std::conditional<F32, int, uint16_t>::type;  // cell type after conversion
  const int nw = blockDim.x >> 5;
  const int L = nw * LW;  // outputs per chunk
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // layout: X[span], Y[span] (type T, then I in place; after the slide the
  // same bytes stage the chunk's L outputs, span >= L), mbarrier, reduction
  // scratch [4][nw]
  T* X = reinterpret_cast<T*>(smem_raw);
  T* Y = X + p.span;
  uint64_t* bar = reinterpret_cast<uint64_t*>(Y + p.span);
  float* red = reinterpret_cast<float*>(bar + 1);
  const I* XI = reinterpret_cast<const I*>(X);
  const I* YI = reinterpret_cast<const I*>(Y);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kAlign = 16 / (int)sizeof(T);  // TMA start coordinate granularity
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    if (p.gx == nullptr) {
      prefetch_tmap(&p.tmx);
      prefetch_tmap(&p.tmy);
    }
  }
  __syncthreads();
  uint32_t phase = 0;
  const int seg = M1 * (UNIT ? 1 : p.stride);
  const int ncell = p.nbox * 256;

  for (long long item = blockIdx.x; item < p.n_items; item += gridDim.x) {
    const long long c0 = item * L;                   // first output of the chunk
    const long long e_first = c0 * p.stride - p.h1;  // first cell of its windows
    const long long e0 = e_first >= 0 ? e_first / kAlign * kAlign : -((-e_first + kAlign - 1) / kAlign) * kAlign;
    const int off = (int)(e_first - e0);             // span offset of cell e_first
    // span cells [v_lo, v_hi) lie on the series
    const int v_lo = (int)max(0ll, -e0);
    const int v_hi = (int)max(0ll, min((long long)ncell, p.N - e0));

    // ---- load the span
    if (p.gx == nullptr) {
      if (tid == 0) mbar_arrive_expect_tx(bar, (uint32_t)(2 * ncell * sizeof(T)));
      __syncthreads();
      for (int b = tid; b < 2 * p.nbox; b += blockDim.x) {
        const bool ych = b >= p.nbox;
        const int bb = ych ? b - p.nbox : b;
        fence_proxy_async_smem();
        tma_load_1d((ych ? Y : X) + (size_t)bb * 256, ych ? &p.tmy : &p.tmx, (int)(e0 + 256ll * bb), bar);
      }
      if (!mbar_wait_bounded(bar, phase, p.status)) return;
      phase ^= 1u;
    } else {
      for (int e = tid; e < ncell; e += blockDim.x) {
        const bool ok = e >= v_lo && e < v_hi;
        X[e] = ok ? reinterpret_cast<const T*>(p.gx)[e0 + e] : (T)0;
        Y[e] = ok ? reinterpret_cast<const T*>(p.gy)[e0 + e] : (T)0;
      }
      __syncthreads();
    }

    // ---- float32: fixed point of the chunk, converted in place
    if constexpr (F32) {
      float xlo = 3.0e38f, xhi = -3.0e38f, ylo = 3.0e38f, yhi = -3.0e38f;
      const float4* X4 = reinterpret_cast<const float4*>(X);
      const float4* Y4 = reinterpret_cast<const float4*>(Y);
      for (int v = tid; v < ncell / 4; v += blockDim.x) {
        const int e = 4 * v;
        const float4 a = X4[v], b = Y4[v];
        if (e >= v_lo && e + 4 <= v_hi) {
          xlo = fminf(xlo, fminf(fminf(a.x, a.y), fminf(a.z, a.w)));
          xhi = fmaxf(xhi, fmaxf(fmaxf(a.x, a.y), fmaxf(a.z, a.w)));
          ylo = fminf(ylo, fminf(fminf(b.x, b.y), fminf(b.z, b.w)));
          yhi = fmaxf(yhi, fmaxf(fmaxf(b.x, b.y), fmaxf(b.z, b.w)));
        } else {
          const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
          for (int u = 0; u < 4; u++)
            if (e + u >= v_lo && e + u < v_hi) {
              xlo = fminf(xlo, av[u]);
              xhi = fmaxf(xhi, av[u]);
              ylo = fminf(ylo, bv[u]);
              yhi = fmaxf(yhi, bv[u]);
            }
        }
      }
      xlo = warp_min(xlo);
      xhi = warp_max(xhi);
      ylo = warp_min(ylo);
      yhi = warp_max(yhi);
      if (lane == 0) {
        red[warp] = xlo;
        red[nw + warp] = xhi;
        red[2 * nw + warp] = ylo;
        red[3 * nw + warp] = yhi;
      }
      __syncthreads();
      xlo = red[0];
      xhi = red[nw];
      ylo = red[2 * nw];
      yhi = red[3 * nw];
      for (int w = 1; w < nw; w++) {
        xlo = fminf(xlo, red[w]);
        xhi = fmaxf(xhi, red[nw + w]);
        ylo = fminf(ylo, red[2 * nw + w]);
        yhi = fmaxf(yhi, red[3 * nw + w]);
      }
      float mx, sx, my, sy;
      fixed_point(xlo, xhi, p.qbits, mx, sx);
      fixed_point(ylo, yhi, p.qbits, my, sy);
      int4* XW = reinterpret_cast<int4*>(X);
      int4* YW = reinterpret_cast<int4*>(Y);
      for (int v = tid; v < ncell / 4; v += blockDim.x) {
        const int e = 4 * v;
        const float4 a = X4[v], b = Y4[v];
        int4 ia = make_int4(to_fixed(a.x, mx, sx), to_fixed(a.y, mx, sx), to_fixed(a.z, mx, sx), to_fixed(a.w, mx, sx));
        int4 ib = make_int4(to_fixed(b.x, my, sy), to_fixed(b.y, my, sy), to_fixed(b.z, my, sy), to_fixed(b.w, my, sy));
        if (!(e >= v_lo && e + 4 <= v_hi)) {
          if (!(e + 0 >= v_lo && e + 0 < v_hi)) ia.x = ib.x = 0;
          if (!(e + 1 >= v_lo && e + 1 < v_hi)) ia.y = ib.y = 0;
          if (!(e + 2 >= v_lo && e + 2 < v_hi)) ia.z = ib.z = 0;
          if (!(e + 3 >= v_lo && e + 3 < v_hi)) ia.w = ib.w = 0;
        }
        XW[v] = ia;
        YW[v] = ib;
      }
      __syncthreads();
    }

    // ---- this warp's outputs: segment sums, first windows, slide
    const int woff = off + warp * LW * p.stride;  // span offset of the warp's first window
    Sums5 Tt[2], R[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
      Tt[h].zero();
      const int g = lane + 32 * h;
      const int b = woff + g * seg;
      // cells past the span never fall inside a window of this chunk
      const int nc = g < p.nseg ? max(0, min(seg, ncell - b)) : 0;
      const int nr = min(p.r, nc);
      int u = 0;
#pragma unroll 4
      for (; u < nr; u++) Tt[h].add((int)XI[b + u], (int)YI[b + u]);
      R[h] = Tt[h];
#pragma unroll 4
      for (; u < nc; u++) Tt[h].add((int)XI[b + u], (int)YI[b + u]);
    }
    // inclusive scan of the 64 segment totals (lanes, then the second half)
    Sums5 C0 = Tt[0], C1 = Tt[1];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const Sums5 a = C0.shfl(max(lane - o, 0)), b = C1.shfl(max(lane - o, 0));
      if (lane >= o) {
        C0.add(a);
        C1.add(b);
      }
    }
    const Sums5 tot0 = C0.shfl(31);
    C1.add(tot0);
    // first window of lane j: segments j .. j+q-1 plus the first r cells of j+q
    // = C(j+q-1) - C(j-1) + R(j+q)
    auto pick_C = [&](int g) -> Sums5 {  // C(g) for g in [-1, 63], uniform-safe shuffles
      Sums5 a = C0.shfl(g & 31), b = C1.shfl(g & 31);
      if (g < 0) {
        a.zero();
        return a;
      }
      return g < 32 ? a : b;
    };
    auto pick_R = [&](int g) -> Sums5 {
      Sums5 a = R[0].shfl(g & 31), b = R[1].shfl(g & 31);
      return g < 32 ? a : b;
    };
    Sums5 W = pick_C(lane + p.q - 1);
    W.sub(pick_C(lane - 1));
    W.add(pick_R(lane + p.q));

    // ---- slide over the lane's outputs (results stay in registers)
    const long long j_base = c0 + (long long)warp * LW + (long long)lane * M1;
    // every window of the lane is whole unless one touches an end of the series
    const bool interior = j_base * p.stride - p.h1 >= 0 && (j_base + M1 - 1) * p.stride + p.h2 <= p.N - 1;
    auto n_of = [&](long long j) -> uint32_t {
      if (interior) return (uint32_t)p.k;
      const long long centre = j * p.stride;
      const long long lo = max(centre - p.h1, 0ll), hi = min(centre + p.h2, p.N - 1);
      return (uint32_t)max(hi - lo + 1, 0ll);
    };
    const int e_out = woff + lane * seg;  // first cell of the lane's first window
    const int e_in = e_out + p.k;         // first cell to enter after it
    float res[M1];
    if constexpr (UNIT) {  // stride 1
#pragma unroll
      for (int t = 0; t < M1; t++) {
        res[t] = pearson_exact(W, n_of(j_base + t));
        if (t + 1 < M1) {
          const int ei = e_in + t, eo = e_out + t;
          const bool in_ok = ei < ncell;
          W.slide(in_ok ? (int)XI[ei] : 0, in_ok ? (int)YI[ei] : 0, (int)XI[eo], (int)YI[eo]);
        }
      }
    } else {
#pragma unroll
      for (int t = 0; t < M1; t++) {
        res[t] = pearson_exact(W, n_of(j_base + t));
        if (t + 1 < M1) {
          for (int u = 0; u < p.stride; u++) {
            const int ei = e_in + t * p.stride + u, eo = e_out + t * p.stride + u;
            const bool in_ok = ei < ncell;
            W.slide(in_ok ? (int)XI[ei] : 0, in_ok ? (int)YI[ei] : 0, (int)XI[eo], (int)YI[eo]);
          }
        }
      }
    }
    // ---- coalesced store of the warp's outputs, staged in the span buffer
    // once every warp of the CTA is done reading it
    __syncthreads();
    float* sw = reinterpret_cast<float*>(X) + warp * LW;
#pragma unroll
    for (int t = 0; t < M1; t++) sw[lane * M1 + t] = res[t];
    __syncwarp();
    const long long wc0 = c0 + (long long)warp * LW;
    const long long nvalid = max(0ll, min((long long)LW, p.n_out - wc0));
    float* dst = p.out + wc0;
    if (nvalid == LW && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
      for (int u = lane; u < LW / 4; u += 32) {
        const float4 v = reinterpret_cast<const float4*>(sw)[u];
        stg128(dst + 4 * u, v.x, v.y, v.z, v.w);
      }
    } else {
      for (int u = lane; u < nvalid; u += 32) dst[u] = sw[u];
    }
    __syncthreads();  // the span is reused by the next chunk
  }
}

}  // namespace swc
