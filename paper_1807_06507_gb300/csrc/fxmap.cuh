// fxmap.cuh -- float32 inputs: the fixed-point map of a block of values, the
// per-window error certificate, and the exact recomputations a window falls
// back to when its certificate fails.
//
// Every float32 kernel maps the values of a block (a 2-D lane's columns over
// its work item, a 1-D chunk, a 3-D work item) to integers
//     X = round((x - m) * s),  s = 2^e,  |X| < 2^q,
// with m on the 2^-e grid (m = M / s, M an integer), and sums them exactly.
// Pearson's c is invariant under this affine map, so the only error is the
// rounding of each value, |X - (x - m) s| <= rho (in units of the grid):
//   * rho = 0 when every value of the block lies on the grid ("exact" block;
//     integer data, or data whose float32 ulp is coarser than 2^-e);
//   * rho = 1/2 when the conversion rounds once: the fused form
//     X = round(x s - M) (one FFMA, |M| <= 2^22), or x - m exact by
//     Sterbenz's lemma (all values of one sign within a factor 2);
//   * rho = 5/8 otherwise (x - m may round by a quarter of the grid step
//     first: |x - m| s < 2^22 gives it an ulp of at most 1/4).
//
// Certificate.  For one window of n cells, let X_c be the centred vector of
// its integers (|X_c|^2 = vx / n, vx = n sum X^2 - (sum X)^2 exact) and e_c
// the centred rounding errors (|e_c| <= rho sqrt(n)).  The angle between X_c
// and the true centred vector is at most asin(z), z = rho n / sqrt(vx), and c
// is the cosine of the angle between the x and y vectors, so
//     |c(X, Y) - c(x, y)| <= asin(z_x) + asin(z_y).
// The kernels' float32 evaluation of Eq. 2 adds at most 7e-7 (relative
// rounding of the int64 -> float32 conversions, the product, rsqrt and the
// final product).  A window is certified when z_x + z_y <= 9e-6, which keeps
// |dc| below 1e-5.  A block with windows that fail is computed again with a
// finer map of the same range (fx_wide: up to 26 bits, 64-bit sums; X =
// round(x s) - M with one rounding, so rho = 1/2 and values on the
// grid convert exactly), certified the same way; a window that still fails
// is recomputed from its own cells with a window-local map of that kind
// (fx_box_exact, fx_box_warp), and, if that fails too, in FP64 in two passes
// (the classical formula, Introduction).
#pragma once

#include <stdint.h>

#include "common.cuh"

namespace swc {

constexpr float kFxMagic = 12582912.0f;  // 1.5 * 2^23: adding it rounds |v| < 2^22 to an integer

struct FxMap {
  float s;     // 2^e (0 maps every value to X = 0: rows outside the grid)
  float C;     // rounding constant: 1.5*2^23 - M in the fused form, 1.5*2^23 otherwise
  float msub;  // subtracted before scaling: 0 in the fused form, m = M / s otherwise
  float rho;   // rounding bound of a value that is not on the grid (1/2 or 5/8)
};

// X = round((x - m) s); one FADD, one FFMA, one IADD.
__device__ __forceinline__ int fx_quant(float x, const FxMap& q) {
  return __float_as_int(fmaf(x - q.msub, q.s, q.C)) - 0x4B400000;
}

// The subtract form with the rounding constant as an immediate.
__device__ __forceinline__ int fx_quant_sub(float x, float msub, float s) {
  return __float_as_int(fmaf(x - msub, s, kFxMagic)) - 0x4B400000;
}

// Map of a block whose values lie in [lo, hi] (lo > hi: no value), q bits.
// The scale leaves a margin of 1/64: A s < 2^q / (1 + 2^-6), so |X| < 0.985 * 2^q
// (the 3-D finalize relies on it) and the fused constant stays exact.
// fused = false keeps the subtract form (C = 1.5*2^23 for every block, one
// register less in a kernel's inner loop).
__device__ __forceinline__ FxMap fx_make(float lo, float hi, int q, bool fused = true) {
  FxMap m;
  if (!(lo <= hi)) lo = hi = 0.0f;
  if (lo == hi) {  // one value: X = 0 for it, exactly
    m.s = 1.0f;
    m.C = kFxMagic;
    m.msub = lo;
    m.rho = 0.5f;
    return m;
  }
  const float mid = lo + 0.5f * (hi - lo);
  const float A = fmaxf(hi - mid, mid - lo);
  int ea;
  frexpf(fmaf(A, 0.015625f, A), &ea);  // A (1 + 2^-6) < 2^ea
  const int e = min(max(q - ea, -126), 126);
  m.s = __int_as_float((127 + e) << 23);
  const float M = rintf(mid * m.s);  // mid * s is exact (power-of-two scale)
  if (fused && fabsf(M) <= 4194304.0f) {
    m.C = kFxMagic - M;  // exact: M is an integer of at most 2^22
    m.msub = 0.0f;
    m.rho = 0.5f;
  } else {
    m.C = kFxMagic;
    m.msub = M * __int_as_float((127 - e) << 23);  // M / s, exact
    // Sterbenz: every x in [lo, hi] and m in it, one sign, within a factor 2
    const bool sterbenz = (lo > 0.0f && hi <= 2.0f * lo) || (hi < 0.0f && lo >= 2.0f * hi);
    m.rho = sterbenz ? 0.5f : 0.625f;
  }
  return m;
}

// True when x converts without rounding: x - msub is exact (TwoSum error 0)
// and (x - msub) s is an integer (the FFMA's rounding error, computed
// exactly, is 0).
__device__ __forceinline__ bool fx_on_grid(float x, const FxMap& q) {
  const float d = x - q.msub;
  const float bv = d - x, av = d - bv;
  const float err = (x - av) + (-q.msub - bv);
  const float t = fmaf(d, q.s, q.C);
  const float K = t - q.C;             // exact: t and C lie in [2^23, 2^24]
  const float r = fmaf(d, q.s, -K);    // d s - K, exactly representable
  return err == 0.0f && r == 0.0f;
}

// Certificate test of one window from its exact integer variances vx, vy
// (n sum X^2 - (sum X)^2, converted to float32 with relative error below
// 2^-21), with per-channel rounding bounds rx, ry.  The float32 evaluation of
// z errs by a few parts in 10^7 of z, inside the margin to 9e-6.
__device__ __forceinline__ bool fx_certified(float vx, float vy, float n, float rx, float ry) {
  if (rx == 0.0f && ry == 0.0f) return true;
  if (!(vx > 0.0f) && rx > 0.0f) return false;
  if (!(vy > 0.0f) && ry > 0.0f) return false;
  const float zx = rx > 0.0f ? rx * n * rsqrtf(vx) : 0.0f;
  const float zy = ry > 0.0f ? ry * n * rsqrtf(vy) : 0.0f;
  return zx + zy <= 8.99e-6f;
}

// int128 -> float32 with relative error below 2^-21 (|v| < 2^95).
__device__ __forceinline__ float i128_to_f32(__int128 v) {
  const long long lo = (long long)v;
  if ((__int128)lo == v) return i64_to_f32(lo);
  return i64_to_f32((long long)(v >> 32)) * 4294967296.0f;
}

// Eq. 2 from exact 128-bit integers in float32 (as the kernels' step 4:
// relative error below 7e-7), clamped; NaN for a zero variance.
__device__ __forceinline__ float fx_pearson128(__int128 num, __int128 vx, __int128 vy) {
  return clamp1_nan(i128_to_f32(num) * rsqrtf(i128_to_f32(vx)) * rsqrtf(i128_to_f32(vy)));
}

// Cells [z0, z1] x [y0, y1] x [x0, x1] (inclusive, inside the grid) of two
// float32 grids with element pitches pz, py.
struct FxBox {
  const float* gx;
  const float* gy;
  long long pz, py;
  int z0, z1, y0, y1, x0, x1;
};

__device__ __forceinline__ int fx_bitlen(unsigned long long v) { return 64 - __clzll(v); }

// Map of a recomputation (window-local, lane-, chunk- or item-wide) of n
// cells whose values lie in [lo, hi], lo < hi: q = min(26, (62 -
// bitlen(n)) / 2) bits (n 2^2q < 2^62 keeps the 64-bit sums of squares
// exact), scale s = 2^e and the integer M = mid s.  A value converts as
// X = round(x s) - M: x s is exact (power-of-two scale), so X is exact when
// x s is an integer (x on the 2^-e grid) and within 1/2 otherwise.  It is
// evaluated in 32 bits.  When |mid| <= 16 A (A the half range), |x s| and
// |M| stay below 17 * 2^26: X = F2I(x s) - M.  Otherwise every x lies within
// A < |mid| / 16 of mid, so x - mid is exact (Sterbenz), mid is on the grid
// (its ulp, at least |mid| 2^-24 > A 2^-20, is a multiple of 2^-e) and
// X = F2I((x - mid) s), the same integer.
struct FxWide {
  float s;
  float sub;  // mid for a block far from 0, else 0
  int moff;   // M for a block near 0, else 0
  long long M;
};
__device__ __forceinline__ FxWide fx_wide(float lo, float hi, long long n) {
  const int q = min(26, (62 - fx_bitlen((unsigned long long)n)) / 2);
  const float mid = lo + 0.5f * (hi - lo);
  const float A = fmaxf(hi - mid, mid - lo);
  int ea;
  frexpf(fmaf(A, 0.015625f, A), &ea);
  const int e = min(max(q - ea, -126), 126);
  FxWide w;
  w.s = __int_as_float((127 + e) << 23);
  w.M = __float2ll_rn(mid * w.s);
  const bool far = fabsf(mid) > 16.0f * A;
  w.sub = far ? mid : 0.0f;
  w.moff = far ? 0 : (int)w.M;
  return w;
}
__device__ __forceinline__ long long fx_wide_quant(float x, const FxWide& w, bool& on_grid) {
  const float v = (x - w.sub) * w.s;  // exact
  on_grid = on_grid && (fabsf(v) >= 8388608.0f || v == rintf(v));
  return (long long)(__float2int_rn(v) - w.moff);
}

// Window-local recomputation: the box's own range and map (fx_wide), exact
// 64-bit sums and Eq. 2 in 128-bit integers.  Returns false if the window's
// certificate fails (the caller then uses fx_box_fp64).
static __device__ __noinline__ bool fx_box_exact(const FxBox& b, float* out) {
  float xlo = 3.0e38f, xhi = -3.0e38f, ylo = 3.0e38f, yhi = -3.0e38f;
  for (int z = b.z0; z <= b.z1; z++)
    for (int y = b.y0; y <= b.y1; y++) {
      const long long o = (long long)z * b.pz + (long long)y * b.py;
#pragma unroll 4
      for (int x = b.x0; x <= b.x1; x++) {
        const float u = b.gx[o + x], v = b.gy[o + x];
        xlo = fminf(xlo, u); xhi = fmaxf(xhi, u); ylo = fminf(ylo, v); yhi = fmaxf(yhi, v);
      }
    }
  if (xlo == xhi || ylo == yhi) {  // a constant channel: zero variance, exactly
    *out = __int_as_float(0x7fc00000);
    return true;
  }
  const long long n = (long long)(b.z1 - b.z0 + 1) * (b.y1 - b.y0 + 1) * (b.x1 - b.x0 + 1);
  const FxWide wx = fx_wide(xlo, xhi, n), wy = fx_wide(ylo, yhi, n);
  long long Sx = 0, Sy = 0, Sxx = 0, Syy = 0, Sxy = 0;
  bool gx_ok = true, gy_ok = true;
  for (int z = b.z0; z <= b.z1; z++)
    for (int y = b.y0; y <= b.y1; y++) {
      const long long o = (long long)z * b.pz + (long long)y * b.py;
#pragma unroll 4
      for (int x = b.x0; x <= b.x1; x++) {
        const long long X = fx_wide_quant(b.gx[o + x], wx, gx_ok), Y = fx_wide_quant(b.gy[o + x], wy, gy_ok);
        Sx += X; Sy += Y; Sxx += X * X; Syy += Y * Y; Sxy += X * Y;
      }
    }
  const __int128 N = n;
  const __int128 vx = N * Sxx - (__int128)Sx * Sx;
  const __int128 vy = N * Syy - (__int128)Sy * Sy;
  const __int128 num = N * Sxy - (__int128)Sx * Sy;
  if (!fx_certified(i128_to_f32(vx), i128_to_f32(vy), (float)n, gx_ok ? 0.0f : 0.5f, gy_ok ? 0.0f : 0.5f))
    return false;
  *out = fx_pearson128(num, vx, vy);  // exact zero variance: NaN
  return true;
}

// FP64 two-pass evaluation of the classical formula (Introduction) over the
// box, with the exact equality test for a constant channel.
static __device__ __noinline__ float fx_box_fp64(const FxBox& b) {
  double sx = 0.0, sy = 0.0;
  const float x00 = b.gx[(long long)b.z0 * b.pz + (long long)b.y0 * b.py + b.x0];
  const float y00 = b.gy[(long long)b.z0 * b.pz + (long long)b.y0 * b.py + b.x0];
  bool cx = true, cy = true;
  for (int z = b.z0; z <= b.z1; z++)
    for (int y = b.y0; y <= b.y1; y++) {
      const long long o = (long long)z * b.pz + (long long)y * b.py;
      for (int x = b.x0; x <= b.x1; x++) {
        const float u = b.gx[o + x], v = b.gy[o + x];
        sx += u; sy += v;
        cx = cx && u == x00; cy = cy && v == y00;
      }
    }
  if (cx || cy) return __int_as_float(0x7fc00000);
  const double n = (double)(b.z1 - b.z0 + 1) * (b.y1 - b.y0 + 1) * (b.x1 - b.x0 + 1);
  const double mx = sx / n, my = sy / n;
  double sxx = 0.0, syy = 0.0, sxy = 0.0;
  for (int z = b.z0; z <= b.z1; z++)
    for (int y = b.y0; y <= b.y1; y++) {
      const long long o = (long long)z * b.pz + (long long)y * b.py;
      for (int x = b.x0; x <= b.x1; x++) {
        const double u = (double)b.gx[o + x] - mx, v = (double)b.gy[o + x] - my;
        sxx += u * u; syy += v * v; sxy += u * v;
      }
    }
  const double cv = sxy / sqrt(sxx * syy);
  return (float)fmin(fmax(cv, -1.0), 1.0);
}

// Warp-cooperative form of fx_box_exact and fx_box_fp64: every lane of a
// warp calls it with the same box.  The box's cells are dealt to the lanes
// (lane l takes cells l, l + 32, ... in x-fastest order), so the loads of one
// step are independent and the window's latency is a few memory round trips
// instead of n; partial ranges and sums are combined by shuffles (exact:
// integer sums).  Returns the window's c in every lane and counts it once.
static __device__ __noinline__ float fx_box_warp(const FxBox& b, uint32_t* status) {
  const int lane = threadIdx.x & 31;
  const int nxb = b.x1 - b.x0 + 1, nyb = b.y1 - b.y0 + 1;
  const long long n = (long long)nxb * nyb * (b.z1 - b.z0 + 1);
  const int dxs = 32 % nxb, dys = 32 / nxb;
  int x0 = lane % nxb, y0 = (lane / nxb) % nyb, z0 = (lane / nxb) / nyb;
  auto advance = [&](int& x, int& y, int& z) {
    x += dxs;
    y += dys;
    if (x >= nxb) {
      x -= nxb;
      y++;
    }
    while (y >= nyb) {
      y -= nyb;
      z++;
    }
  };
  auto offset = [&](int x, int y, int z) {
    return (long long)(b.z0 + z) * b.pz + (long long)(b.y0 + y) * b.py + b.x0 + x;
  };
  float xlo = 3.0e38f, xhi = -3.0e38f, ylo = 3.0e38f, yhi = -3.0e38f;
  {
    int x = x0, y = y0, z = z0;
    for (long long i = lane; i < n; i += 32) {
      const long long o = offset(x, y, z);
      const float u = b.gx[o], v = b.gy[o];
      xlo = fminf(xlo, u); xhi = fmaxf(xhi, u); ylo = fminf(ylo, v); yhi = fmaxf(yhi, v);
      advance(x, y, z);
    }
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    xlo = fminf(xlo, __shfl_xor_sync(0xffffffffu, xlo, d));
    xhi = fmaxf(xhi, __shfl_xor_sync(0xffffffffu, xhi, d));
    ylo = fminf(ylo, __shfl_xor_sync(0xffffffffu, ylo, d));
    yhi = fmaxf(yhi, __shfl_xor_sync(0xffffffffu, yhi, d));
  }
  float c;
  if (xlo == xhi || ylo == yhi) {  // a constant channel: zero variance, exactly
    c = __int_as_float(0x7fc00000);
  } else {
    const FxWide wx = fx_wide(xlo, xhi, n), wy = fx_wide(ylo, yhi, n);
    long long S[5] = {0, 0, 0, 0, 0};
    bool okx = true, oky = true;
    {
      int x = x0, y = y0, z = z0;
      for (long long i = lane; i < n; i += 32) {
        const long long o = offset(x, y, z);
        const long long X = fx_wide_quant(b.gx[o], wx, okx), Y = fx_wide_quant(b.gy[o], wy, oky);
        S[0] += X; S[1] += Y; S[2] += X * X; S[3] += Y * Y; S[4] += X * Y;
        advance(x, y, z);
      }
    }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1)
#pragma unroll
      for (int t = 0; t < 5; t++) S[t] += __shfl_xor_sync(0xffffffffu, S[t], d);
    okx = __all_sync(0xffffffffu, okx);
    oky = __all_sync(0xffffffffu, oky);
    const __int128 N = n;
    const __int128 vx = N * S[2] - (__int128)S[0] * S[0];
    const __int128 vy = N * S[3] - (__int128)S[1] * S[1];
    const __int128 num = N * S[4] - (__int128)S[0] * S[1];
    if (fx_certified(i128_to_f32(vx), i128_to_f32(vy), (float)n, okx ? 0.0f : 0.5f, oky ? 0.0f : 0.5f)) {
      c = fx_pearson128(num, vx, vy);
    } else {  // FP64, two passes (the classical formula, Introduction)
      double sx = 0.0, sy = 0.0;
      {
        int x = x0, y = y0, z = z0;
        for (long long i = lane; i < n; i += 32) {
          const long long o = offset(x, y, z);
          sx += b.gx[o];
          sy += b.gy[o];
          advance(x, y, z);
        }
      }
#pragma unroll
      for (int d = 16; d >= 1; d >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, d);
        sy += __shfl_xor_sync(0xffffffffu, sy, d);
      }
      const double mx = sx / (double)n, my = sy / (double)n;
      double sxx = 0.0, syy = 0.0, sxy = 0.0;
      {
        int x = x0, y = y0, z = z0;
        for (long long i = lane; i < n; i += 32) {
          const long long o = offset(x, y, z);
          const double u = (double)b.gx[o] - mx, v = (double)b.gy[o] - my;
          sxx += u * u; syy += v * v; sxy += u * v;
          advance(x, y, z);
        }
      }
#pragma unroll
      for (int d = 16; d >= 1; d >>= 1) {
        sxx += __shfl_xor_sync(0xffffffffu, sxx, d);
        syy += __shfl_xor_sync(0xffffffffu, syy, d);
        sxy += __shfl_xor_sync(0xffffffffu, sxy, d);
      }
      c = (float)fmin(fmax(sxy / sqrt(sxx * syy), -1.0), 1.0);
    }
  }
  if (lane == 0 && status) atomicAdd(status + ST_FALLBACK, 1u);
  return c;
}

}  // namespace swc
