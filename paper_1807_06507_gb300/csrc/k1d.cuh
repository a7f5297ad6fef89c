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
//    float32 through a fixed-point map of the chunk (fxmap.cuh: reference on
//    the grid near the midpoint of the chunk's range, power-of-two scale,
//    |X| < 2^qbits with n 2^qbits < 2^31), converted in place four cells per
//    access, noting whether every value converted without rounding.  Cells
//    off the series become 0.
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
//  * float32 certificate (fxmap.cuh): a window passes when
//    vx, vy >= (rho n / 4.5e-6)^2 (rho = 0 for a channel whose chunk
//    converted exactly).  A chunk with failing windows is listed; a second
//    launch of this kernel in its wide form runs the listed chunks again
//    with a map of up to 26 bits of the chunk's range (fx_wide), 64-bit
//    first moments and Eq. 2 in 128-bit integers, rewriting every output of
//    the chunk.  A lane whose windows still fail recomputes them from the
//    chunk's floats with a map of its own span, sliding from window to
//    window; a window that fails that too is recomputed from its own cells.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "fxmap.cuh"
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

// The wide form's window sums: 64-bit first moments (values of up to 26
// bits, fx_wide), all modular.
struct Sums5W {
  uint64_t x, y, xx, yy, xy;
  __device__ __forceinline__ void zero() { x = y = xx = yy = xy = 0ull; }
  __device__ __forceinline__ void add(int X, int Y) {
    x += (uint64_t)(long long)X;
    y += (uint64_t)(long long)Y;
    xx += (uint64_t)((long long)X * X);
    yy += (uint64_t)((long long)Y * Y);
    xy += (uint64_t)((long long)X * Y);
  }
  __device__ __forceinline__ void slide(int Xi, int Yi, int Xo, int Yo) {
    const int dx = Xi - Xo, dy = Yi - Yo;
    x += (uint64_t)(long long)dx;
    y += (uint64_t)(long long)dy;
    xx += (uint64_t)((long long)dx * (Xi + Xo));
    yy += (uint64_t)((long long)dy * (Yi + Yo));
    xy += (uint64_t)((long long)dx * Yi + (long long)Xo * dy);
  }
  __device__ __forceinline__ void add(const Sums5W& o) { x += o.x; y += o.y; xx += o.xx; yy += o.yy; xy += o.xy; }
  __device__ __forceinline__ void sub(const Sums5W& o) { x -= o.x; y -= o.y; xx -= o.xx; yy -= o.yy; xy -= o.xy; }
  __device__ __forceinline__ Sums5W shfl(int src) const {
    Sums5W r;
    r.x = __shfl_sync(0xffffffffu, x, src);
    r.y = __shfl_sync(0xffffffffu, y, src);
    r.xx = __shfl_sync(0xffffffffu, xx, src);
    r.yy = __shfl_sync(0xffffffffu, yy, src);
    r.xy = __shfl_sync(0xffffffffu, xy, src);
    return r;
  }
};

// Eq. 2 of the wide form in 128-bit integers (sums of X^2 below 2^62), with
// the precise certificate (rx, ry: the channels' rounding bounds).
__device__ __forceinline__ float pearson_wide(const Sums5W& s, uint32_t n, float rx, float ry, bool& fail) {
  const __int128 N = n;
  const long long sx = (long long)s.x, sy = (long long)s.y;
  const __int128 vx = N * (long long)s.xx - (__int128)sx * sx;
  const __int128 vy = N * (long long)s.yy - (__int128)sy * sy;
  const __int128 num = N * (long long)s.xy - (__int128)sx * sy;
  fail = !fx_certified(i128_to_f32(vx), i128_to_f32(vy), (float)n, rx, ry);
  return fx_pearson128(num, vx, vy);
}

// Eq. 2 from exact modular window sums (the results fit in int64; the first
// moments are below 2^31 in magnitude).  fail: the float32 certificate's
// quick test (vx >= Kx, vy >= Ky) did not pass.
__device__ __forceinline__ float pearson_exact(const Sums5& s, uint32_t n, float Kx, float Ky, bool& fail) {
  const long long sx = (int)s.x, sy = (int)s.y;
  const long long vx = (long long)((uint64_t)n * s.xx - (uint64_t)(sx * sx));
  const long long vy = (long long)((uint64_t)n * s.yy - (uint64_t)(sy * sy));
  const long long num = (long long)((uint64_t)n * s.xy - (uint64_t)(sx * sy));
  const float fvx = i64_to_f32(vx), fvy = i64_to_f32(vy);
  fail = !(fvx >= Kx && fvy >= Ky);
  // a zero variance makes num exactly 0, so 0 * rsqrt(0) = NaN
  return clamp1_nan(i64_to_f32(num) * rsqrtf(fvx * fvy));
}

// Debug output of uint16 plans: the exact window sums of output j.
__device__ __forceinline__ void emit_sums(const K1DParams& p, const Sums5& W, long long j) {
  if (p.sums != nullptr && j < p.n_out) {
    long long* s5 = p.sums + 5 * j;
    s5[0] = (int)W.x;  // below 2^31 for uint16 windows of at most 32768 cells
    s5[1] = (int)W.y;
    s5[2] = (long long)W.xx;
    s5[3] = (long long)W.yy;
    s5[4] = (long long)W.xy;
  }
}

// Recompute the failing outputs (bits of `fail`) of one lane whose first
// output is j_base, from the chunk's float32 span in shared memory (cell i of
// the series at gx[i - e0]): a fixed-point map of the lane's own span
// (fx_wide: up to 26 bits, exact for values on the grid, else within 1/2),
// 64-bit window sums slid from one failing window to the next, Eq. 2 in
// 128-bit integers, the certificate;
// windows that still fail are recomputed from their cells.  Writes out[j]
// directly and counts every recomputed window.
static __device__ __noinline__ void lane_redo_1d(const float* sx_span, const float* sy_span, long long e0,
                                                 long long N, int k, int h1, int h2, int stride, long long j_base,
                                                 uint64_t fail, long long n_out, float* out, uint32_t* status) {
  const float* gx = sx_span - e0;  // indexed by series cell (every cell used lies in the span)
  const float* gy = sy_span - e0;
  const int ta = __ffsll((long long)fail) - 1, tb = 63 - __clzll((long long)fail);
  const long long a = max(0ll, (j_base + ta) * stride - h1), b = min(N - 1, (j_base + tb) * stride + h2);
  // range of the span: four independent accumulators (the loop is latency-bound)
  float rlo[4] = {3.0e38f, 3.0e38f, 3.0e38f, 3.0e38f}, rhi[4] = {-3.0e38f, -3.0e38f, -3.0e38f, -3.0e38f};
  float slo[4] = {3.0e38f, 3.0e38f, 3.0e38f, 3.0e38f}, shi[4] = {-3.0e38f, -3.0e38f, -3.0e38f, -3.0e38f};
  for (long long i = a; i <= b; i += 4) {
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const long long iu = min(i + u, b);
      const float p = gx[iu], v = gy[iu];
      rlo[u] = fminf(rlo[u], p); rhi[u] = fmaxf(rhi[u], p); slo[u] = fminf(slo[u], v); shi[u] = fmaxf(shi[u], v);
    }
  }
  const float xlo = fminf(fminf(rlo[0], rlo[1]), fminf(rlo[2], rlo[3]));
  const float xhi = fmaxf(fmaxf(rhi[0], rhi[1]), fmaxf(rhi[2], rhi[3]));
  const float ylo = fminf(fminf(slo[0], slo[1]), fminf(slo[2], slo[3]));
  const float yhi = fmaxf(fmaxf(shi[0], shi[1]), fmaxf(shi[2], shi[3]));
  if (xlo == xhi || ylo == yhi) {  // a channel whose span is one value: every window is constant
    uint32_t count = 0;
    for (int t = ta; t <= tb; t++)
      if (((fail >> t) & 1ull) && j_base + t < n_out) {
        out[j_base + t] = __int_as_float(0x7fc00000);
        count++;
      }
    if (count) atomicAdd(status + ST_FALLBACK, count);
    return;
  }
  const FxWide wx = fx_wide(xlo, xhi, k), wy = fx_wide(ylo, yhi, k);
  long long Sx = 0, Sy = 0, Sxx = 0, Syy = 0, Sxy = 0;
  bool gx_ok = true, gy_ok = true;  // every value read so far on its channel's grid
  auto cell = [&](long long i, int sign) {
    const long long X = fx_wide_quant(gx[i], wx, gx_ok), Y = fx_wide_quant(gy[i], wy, gy_ok);
    Sx += sign * X; Sy += sign * Y; Sxx += sign * (X * X); Syy += sign * (Y * Y); Sxy += sign * (X * Y);
  };
  long long lo = 0, hi = -1;  // cells currently summed
  uint32_t count = 0;
  for (int t = ta; t <= tb; t++) {
    if (!((fail >> t) & 1ull)) continue;
    const long long j = j_base + t;
    if (j >= n_out) break;
    const long long nlo = max(0ll, j * stride - h1), nhi = min(N - 1, j * stride + h2);
    if (nlo > hi) {  // no overlap with the previous window: start again, four partial sums at a time
      long long p[4][5] = {};
      bool okx = true, oky = true;
      long long i = nlo;
      for (; i + 3 <= nhi; i += 4) {
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const long long X = fx_wide_quant(gx[i + u], wx, okx), Y = fx_wide_quant(gy[i + u], wy, oky);
          p[u][0] += X; p[u][1] += Y; p[u][2] += X * X; p[u][3] += Y * Y; p[u][4] += X * Y;
        }
      }
      gx_ok = gx_ok && okx;
      gy_ok = gy_ok && oky;
      Sx = p[0][0] + p[1][0] + p[2][0] + p[3][0];
      Sy = p[0][1] + p[1][1] + p[2][1] + p[3][1];
      Sxx = p[0][2] + p[1][2] + p[2][2] + p[3][2];
      Syy = p[0][3] + p[1][3] + p[2][3] + p[3][3];
      Sxy = p[0][4] + p[1][4] + p[2][4] + p[3][4];
      for (; i <= nhi; i++) cell(i, 1);
    } else {
      for (long long i = lo; i < nlo; i++) cell(i, -1);
      for (long long i = hi + 1; i <= nhi; i++) cell(i, 1);
    }
    lo = nlo;
    hi = nhi;
    const long long n = nhi - nlo + 1;
    const __int128 vx = (__int128)n * Sxx - (__int128)Sx * Sx;
    const __int128 vy = (__int128)n * Syy - (__int128)Sy * Sy;
    const __int128 num = (__int128)n * Sxy - (__int128)Sx * Sy;
    float c;
    if (fx_certified(i128_to_f32(vx), i128_to_f32(vy), (float)n, gx_ok ? 0.0f : 0.5f, gy_ok ? 0.0f : 0.5f)) {
      c = fx_pearson128(num, vx, vy);  // exact zero variance: NaN
    } else {
      FxBox bx;
      bx.gx = sx_span;
      bx.gy = sy_span;
      bx.pz = bx.py = 0;
      bx.z0 = bx.z1 = bx.y0 = bx.y1 = 0;
      bx.x0 = (int)(nlo - e0);
      bx.x1 = (int)(nhi - e0);
      if (!fx_box_exact(bx, &c)) c = fx_box_fp64(bx);
    }
    out[j] = c;
    count++;
  }
  if (count) atomicAdd(status + ST_FALLBACK, count);
}

// WIDE = true (float32 only): the second tier, run on the chunks the first
// launch listed, with a map of up to 26 bits of the chunk's range (fx_wide),
// 64-bit first moments and Eq. 2 in 128-bit integers.
template <int M1, bool F32, bool UNIT, bool WIDE>
__global__ void __launch_bounds__(128, 3) k1d_kernel(const __grid_constant__ K1DParams p) {
  static_assert(F32 || !WIDE, "the wide form is float32 only");
  using S5 = std::conditional_t<WIDE, Sums5W, Sums5>;
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

  const long long n_iter = WIDE ? (long long)*p.redo_count : p.n_items;
  for (long long it = blockIdx.x; it < n_iter; it += gridDim.x) {
    const long long item = WIDE ? p.redo_items[it] : it;
    const long long c0 = item * L;                   // first output of the chunk
    const long long e_first = c0 * p.stride - p.h1;  // first cell of its windows
    const long long e0 = e_first >= 0 ? e_first / kAlign * kAlign : -((-e_first + kAlign - 1) / kAlign) * kAlign;
    const int off = (int)(e_first - e0);             // span offset of cell e_first
    // span cells [v_lo, v_hi) lie on the series
    const int v_lo = (int)max(0ll, -e0);
    const int v_hi = (int)max(0ll, min((long long)ncell, p.N - e0));

    // ---- load the span
    auto load_span = [&]() -> bool {
      if (p.gx == nullptr) {
        if (tid == 0) mbar_arrive_expect_tx(bar, (uint32_t)(2 * ncell * sizeof(T)));
        __syncthreads();
        for (int b = tid; b < 2 * p.nbox; b += blockDim.x) {
          const bool ych = b >= p.nbox;
          const int bb = ych ? b - p.nbox : b;
          fence_proxy_async_smem();
          tma_load_1d((ych ? Y : X) + (size_t)bb * 256, ych ? &p.tmy : &p.tmx, (int)(e0 + 256ll * bb), bar);
        }
        if (!mbar_wait_bounded(bar, phase, p.status)) return false;
        phase ^= 1u;
      } else {
        for (int e = tid; e < ncell; e += blockDim.x) {
          const bool ok = e >= v_lo && e < v_hi;
          X[e] = ok ? reinterpret_cast<const T*>(p.gx)[e0 + e] : (T)0;
          Y[e] = ok ? reinterpret_cast<const T*>(p.gy)[e0 + e] : (T)0;
        }
        __syncthreads();
      }
      return true;
    };
    if (!load_span()) return;

    // ---- float32: fixed point of the chunk, converted in place
    float Kx = 0.0f, Ky = 0.0f;  // certificate thresholds (0: exact, or uint16)
    float wrx = 0.0f, wry = 0.0f;  // wide form: rounding bounds (0: every value on the grid)
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
      int4* XW = reinterpret_cast<int4*>(X);
      int4* YW = reinterpret_cast<int4*>(Y);
      if constexpr (WIDE) {
        // X = round(x s) - M, one rounding (fx_wide)
        const FxWide wx = fx_wide(xlo, xhi, p.k), wy = fx_wide(ylo, yhi, p.k);
        const bool const_ch = !(xlo < xhi) || !(ylo < yhi);  // a constant channel: every window NaN
        bool gx = true, gy = true;
        for (int v = tid; v < ncell / 4; v += blockDim.x) {
          const int e = 4 * v;
          const float4 a = X4[v], b = Y4[v];
          const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
          int ia[4], ib[4];
#pragma unroll
          for (int u = 0; u < 4; u++) {
            const bool on = !const_ch && e + u >= v_lo && e + u < v_hi;
            ia[u] = on ? (int)fx_wide_quant(av[u], wx, gx) : 0;
            ib[u] = on ? (int)fx_wide_quant(bv[u], wy, gy) : 0;
          }
          XW[v] = make_int4(ia[0], ia[1], ia[2], ia[3]);
          YW[v] = make_int4(ib[0], ib[1], ib[2], ib[3]);
        }
        wrx = __syncthreads_or(!gx) ? 0.5f : 0.0f;
        wry = __syncthreads_or(!gy) ? 0.5f : 0.0f;
      } else {
      const FxMap qx = fx_make(xlo, xhi, p.qbits), qy = fx_make(ylo, yhi, p.qbits);
      // conversion in place; rx, ry: largest rounding residual of an on-series value
      float rx = 0.0f, ry = 0.0f;
      auto cv = [&](float v, const FxMap& q, float& racc, bool on) {
        const float d = v - q.msub;
        const float t = fmaf(d, q.s, q.C);
        const float r = fmaf(d, q.s, -(t - q.C));  // the conversion's rounding, exactly
        racc = on ? fmaxf(racc, fabsf(r)) : racc;
        return on ? __float_as_int(t) - 0x4B400000 : 0;
      };
      for (int v = tid; v < ncell / 4; v += blockDim.x) {
        const int e = 4 * v;
        const float4 a = X4[v], b = Y4[v];
        int4 ia, ib;
        if (e >= v_lo && e + 4 <= v_hi) {
          ia = make_int4(cv(a.x, qx, rx, true), cv(a.y, qx, rx, true), cv(a.z, qx, rx, true), cv(a.w, qx, rx, true));
          ib = make_int4(cv(b.x, qy, ry, true), cv(b.y, qy, ry, true), cv(b.z, qy, ry, true), cv(b.w, qy, ry, true));
        } else {
          const bool o0 = e >= v_lo && e < v_hi, o1 = e + 1 >= v_lo && e + 1 < v_hi;
          const bool o2 = e + 2 >= v_lo && e + 2 < v_hi, o3 = e + 3 >= v_lo && e + 3 < v_hi;
          ia = make_int4(cv(a.x, qx, rx, o0), cv(a.y, qx, rx, o1), cv(a.z, qx, rx, o2), cv(a.w, qx, rx, o3));
          ib = make_int4(cv(b.x, qy, ry, o0), cv(b.y, qy, ry, o1), cv(b.z, qy, ry, o2), cv(b.w, qy, ry, o3));
        }
        XW[v] = ia;
        YW[v] = ib;
      }
      // a channel converts exactly when no value rounded and x - m is exact
      // (fused form, or one sign within a factor 2: rho = 1/2)
      const bool inexact_x = __syncthreads_or(rx != 0.0f) || qx.rho != 0.5f;
      const bool inexact_y = __syncthreads_or(ry != 0.0f) || qy.rho != 0.5f;
      const float k0 = 4.9432e10f * (float)p.k * (float)p.k;  // (1 / 4.5e-6)^2 * 1.001 * n^2
      Kx = inexact_x ? k0 * qx.rho * qx.rho : 0.0f;
      Ky = inexact_y ? k0 * qy.rho * qy.rho : 0.0f;
      }
    }

    // ---- this warp's outputs: segment sums, first windows, slide
    const int woff = off + warp * LW * p.stride;  // span offset of the warp's first window
    S5 Tt[2], R[2];
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
    S5 C0 = Tt[0], C1 = Tt[1];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const S5 a = C0.shfl(max(lane - o, 0)), b = C1.shfl(max(lane - o, 0));
      if (lane >= o) {
        C0.add(a);
        C1.add(b);
      }
    }
    const S5 tot0 = C0.shfl(31);
    C1.add(tot0);
    // first window of lane j: segments j .. j+q-1 plus the first r cells of j+q
    // = C(j+q-1) - C(j-1) + R(j+q)
    auto pick_C = [&](int g) -> S5 {  // C(g) for g in [-1, 63], uniform-safe shuffles
      S5 a = C0.shfl(g & 31), b = C1.shfl(g & 31);
      if (g < 0) {
        a.zero();
        return a;
      }
      return g < 32 ? a : b;
    };
    auto pick_R = [&](int g) -> S5 {
      S5 a = R[0].shfl(g & 31), b = R[1].shfl(g & 31);
      return g < 32 ? a : b;
    };
    S5 W = pick_C(lane + p.q - 1);
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
    uint64_t fail = 0;  // outputs whose certificate's quick test failed
    // the wide form runs on a few chunks per launch: a rolled slide keeps its
    // 128-bit finalize from filling a cold instruction cache
    constexpr int kSlideUnroll = WIDE ? 1 : M1;
    if constexpr (UNIT) {  // stride 1
#pragma unroll kSlideUnroll
      for (int t = 0; t < M1; t++) {
        bool f;
        if constexpr (WIDE)
          res[t] = pearson_wide(W, n_of(j_base + t), wrx, wry, f);
        else
          res[t] = pearson_exact(W, n_of(j_base + t), Kx, Ky, f);
        fail |= (uint64_t)f << t;
        if constexpr (!F32) emit_sums(p, W, j_base + t);
        if (t + 1 < M1) {
          const int ei = e_in + t, eo = e_out + t;
          const bool in_ok = ei < ncell;
          W.slide(in_ok ? (int)XI[ei] : 0, in_ok ? (int)YI[ei] : 0, (int)XI[eo], (int)YI[eo]);
        }
      }
    } else {
#pragma unroll kSlideUnroll
      for (int t = 0; t < M1; t++) {
        bool f;
        if constexpr (WIDE)
          res[t] = pearson_wide(W, n_of(j_base + t), wrx, wry, f);
        else
          res[t] = pearson_exact(W, n_of(j_base + t), Kx, Ky, f);
        fail |= (uint64_t)f << t;
        if constexpr (!F32) emit_sums(p, W, j_base + t);
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
#pragma unroll kSlideUnroll
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
    if constexpr (WIDE) {
      // every output of the chunk was rewritten; lanes with windows that
      // still fail recompute them from the chunk's floats, loaded again into
      // the span buffer once every warp has stored
      if (lane == 0 && nvalid > 0) atomicAdd(p.status + ST_FALLBACK, (uint32_t)nvalid);
      if (__syncthreads_or(fail != 0ull)) {
        if (!load_span()) return;
        if (fail)
          lane_redo_1d(reinterpret_cast<const float*>(X), reinterpret_cast<const float*>(Y), e0, p.N, p.k, p.h1, p.h2,
                       p.stride, j_base, fail, p.n_out, p.out, p.status);
      }
    } else if constexpr (F32) {
      // a chunk with failing windows (its values do not all convert exactly,
      // or no window could fail) is listed for the wide launch
      if (__syncthreads_or(fail != 0ull) && tid == 0) p.redo_items[atomicAdd(p.redo_count, 1)] = item;
    }
    __syncthreads();  // the span is reused by the next chunk
  }
}

}  // namespace swc
