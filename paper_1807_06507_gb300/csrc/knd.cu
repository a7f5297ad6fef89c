// knd.cu -- the general n-dimensional path (1 to 8 dimensions).
//
// The optimized algorithm in the form the paper states it (Section 1,
// steps 1-4 and the n-dimensional generalisation; Section 2 runs each step
// as one parallel phase): the five products are materialised as integer
// streams, each dimension gets one sliding-sum pass over them, and Eq. 2 is
// evaluated from the resulting window sums.  It serves what the fused
// kernels do not: grids of more than three dimensions, the paper's -2 result
// convention (Section 3, the result-set paragraph) and, as an ablation, the
// cumulative-sum alternative the paper rejects (Section 1, last paragraph).
//
//  * Streams (int64, structure of arrays over the grid's cells in C order):
//    X, Y, X^2, Y^2, XY and, for the -2 convention, the count of missing
//    cells (a value <= -999 in x or y; such a cell adds 0 to the others).
//    uint16 cells are X = x; float32 cells go through one fixed-point map of
//    the whole grid (fxmap.cuh) taken from a range pass, with the same
//    certificate as the fused kernels; a window that fails it is recomputed
//    from its own cells with a window-local map (26 bits, exact 64-bit sums),
//    and in FP64 if that fails too.  All sums are exact (modular) integers.
//  * Pass along dimension d: sliding sums over the clipped window
//    [i - floor((k-1)/2), i + floor(k/2)] (outside cells add nothing); one
//    thread per segment of a line (a running sum) for the outer dimensions,
//    one thread per cell for the contiguous one.  The cumulative-sum ablation instead
//    takes inclusive prefix sums along every dimension (modulo 2^64, still
//    exact) and forms each window by inclusion-exclusion over its 2^ndim
//    corners.
//  * Finalize: n is the product of the clipped extents; -2 for a window past
//    an edge or with a missing cell under the paper's convention; Eq. 2 in
//    128-bit integers, one float32 rounding per factor; NaN for a zero
//    variance; clamp to [-1, 1].
//  * Mask-only form: after a fused kernel has written every window with
//    clipped borders, the paper's convention needs only the -2 outputs: one
//    stream (the missing-cell count, float32 only), its sliding sums, and a
//    finalize that writes -2 and nothing else (a window that neither passes
//    an edge nor holds a missing cell is whole, so the fused result is the
//    convention's result).
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "fxmap.cuh"
#include "knd.h"

namespace swc {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int ord_of(float f) {  // order-preserving int of a float
  const int i = __float_as_int(f);
  return i ^ ((i >> 31) & 0x7fffffff);
}
__device__ __forceinline__ float float_of(int i) { return __int_as_float(i ^ ((i >> 31) & 0x7fffffff)); }

// input offset of flat cell index `cell` (C order over shape)
__device__ __forceinline__ long long in_offset(const KNDParams& p, long long cell) {
  long long off = 0;
  for (int d = p.ndim - 1; d >= 0; d--) {
    const long long i = cell % p.shape[d];
    cell /= p.shape[d];
    off += i * p.ipitch[d];
  }
  return off;
}

__device__ __forceinline__ void load_cell(const KNDParams& p, long long off, float& a, float& b) {
  if (p.is_f32) {
    a = ((const float*)p.x)[off];
    b = ((const float*)p.y)[off];
  } else {
    a = (float)((const uint16_t*)p.x)[off];
    b = (float)((const uint16_t*)p.y)[off];
  }
}

__device__ __forceinline__ FxMap map_of(const KNDParams& p, int ch) {
  const int* r = reinterpret_cast<const int*>(p.scratch);
  return fx_make(float_of(r[2 * ch]), float_of(r[2 * ch + 1]), p.qbits);
}

__global__ void nd_init(KNDParams p) {
  int* r = reinterpret_cast<int*>(p.scratch);
  r[0] = r[2] = 0x7fffffff;  // min of x, y (order-preserving ints)
  r[1] = r[3] = (int)0x80000000;  // max
  r[4] = 0;  // some value does not convert exactly
}

__global__ void __launch_bounds__(kThreads) nd_range(KNDParams p) {
  int lo0 = 0x7fffffff, hi0 = (int)0x80000000, lo1 = 0x7fffffff, hi1 = (int)0x80000000;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < p.ncell; c += (long long)gridDim.x * blockDim.x) {
    float a, b;
    load_cell(p, in_offset(p, c), a, b);
    if (p.paper && (a <= -999.0f || b <= -999.0f)) continue;
    lo0 = min(lo0, ord_of(a)); hi0 = max(hi0, ord_of(a));
    lo1 = min(lo1, ord_of(b)); hi1 = max(hi1, ord_of(b));
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo0 = min(lo0, __shfl_xor_sync(0xffffffffu, lo0, o));
    hi0 = max(hi0, __shfl_xor_sync(0xffffffffu, hi0, o));
    lo1 = min(lo1, __shfl_xor_sync(0xffffffffu, lo1, o));
    hi1 = max(hi1, __shfl_xor_sync(0xffffffffu, hi1, o));
  }
  if ((threadIdx.x & 31) == 0) {
    int* r = reinterpret_cast<int*>(p.scratch);
    atomicMin(r + 0, lo0); atomicMax(r + 1, hi0); atomicMin(r + 2, lo1); atomicMax(r + 3, hi1);
  }
}

__global__ void __launch_bounds__(kThreads) nd_convert(KNDParams p) {
  long long* S = p.buf[0];
  FxMap qx{}, qy{};
  if (p.is_f32) {
    qx = map_of(p, 0);
    qy = map_of(p, 1);
  }
  bool inexact = false;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < p.ncell; c += (long long)gridDim.x * blockDim.x) {
    float a, b;
    load_cell(p, in_offset(p, c), a, b);
    const bool miss = p.paper && (a <= -999.0f || b <= -999.0f);
    if (p.mask_only) {
      S[c] = miss ? 1 : 0;
      continue;
    }
    long long X = 0, Y = 0;
    if (!miss) {
      if (p.is_f32) {
        X = fx_quant(a, qx);
        Y = fx_quant(b, qy);
        inexact = inexact || !fx_on_grid(a, qx) || !fx_on_grid(b, qy);
      } else {
        X = (long long)a;
        Y = (long long)b;
      }
    }
    S[c] = X;
    S[p.ncell + c] = Y;
    S[2 * p.ncell + c] = X * X;
    S[3 * p.ncell + c] = Y * Y;
    S[4 * p.ncell + c] = X * Y;
    if (p.nstreams > 5) S[5 * p.ncell + c] = miss ? 1 : 0;
  }
  if (__any_sync(0xffffffffu, inexact) && (threadIdx.x & 31) == 0) atomicOr(reinterpret_cast<int*>(p.scratch) + 4, 1);
}

// Pass along an outer dimension d (cells of a line are inner[d] apart).  A
// line is cut into segments of kSeg cells, one thread each (threads of a
// warp take neighbouring lines, so their accesses are contiguous): sliding
// sums start each segment with its first window summed directly; the
// cumulative-sum ablation takes segment totals, scans them per line, then
// writes each segment's prefix from its offset.
constexpr int kSeg = 128;

__device__ __forceinline__ void seg_of(const KNDParams& p, int d, long long t, long long& base, long long& i0,
                                       long long& i1) {
  const long long N = p.shape[d], step = p.inner[d];
  const long long nseg = (N + kSeg - 1) / kSeg, lines = p.ncell / N;
  const long long line = t % lines, seg = t / lines;
  base = (line / step) * N * step + line % step;
  i0 = seg * kSeg;
  i1 = min(N, i0 + kSeg);
  (void)nseg;
}

__global__ void __launch_bounds__(kThreads) nd_pass_lines(KNDParams p, int d, const long long* in, long long* out) {
  const long long N = p.shape[d], step = p.inner[d];
  const long long total = (p.ncell / N) * ((N + kSeg - 1) / kSeg);
  const int h1 = p.h1[d], h2 = p.h2[d];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    long long base, i0, i1;
    seg_of(p, d, t, base, i0, i1);
    for (int s = 0; s < p.nstreams; s++) {
      const long long* src = in + s * p.ncell + base;
      long long* dst = out + s * p.ncell + base;
      unsigned long long acc = 0;
      for (long long i = max(0ll, i0 - h1); i <= min(N - 1, i0 + (long long)h2); i++) acc += (unsigned long long)src[i * step];
      for (long long i = i0; i < i1; i++) {
        dst[i * step] = (long long)acc;
        if (i + h2 + 1 < N) acc += (unsigned long long)src[(i + h2 + 1) * step];
        if (i - h1 >= 0) acc -= (unsigned long long)src[(i - h1) * step];
      }
    }
  }
}

// cumulative sums along an outer dimension: (1) segment totals into seg[]
__global__ void __launch_bounds__(kThreads) nd_scan_lines_totals(KNDParams p, int d, const long long* in) {
  const long long N = p.shape[d], step = p.inner[d];
  const long long total = (p.ncell / N) * ((N + kSeg - 1) / kSeg);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    long long base, i0, i1;
    seg_of(p, d, t, base, i0, i1);
    for (int s = 0; s < p.nstreams; s++) {
      unsigned long long acc = 0;
      for (long long i = i0; i < i1; i++) acc += (unsigned long long)in[s * p.ncell + base + i * step];
      p.segs[s * total + t] = (long long)acc;
    }
  }
}

// (2) exclusive scan of each line's segment totals (one thread per line)
__global__ void __launch_bounds__(kThreads) nd_scan_lines_offsets(KNDParams p, int d) {
  const long long N = p.shape[d], lines = p.ncell / N, nseg = (N + kSeg - 1) / kSeg, total = lines * nseg;
  for (long long line = blockIdx.x * (long long)blockDim.x + threadIdx.x; line < lines;
       line += (long long)gridDim.x * blockDim.x)
    for (int s = 0; s < p.nstreams; s++) {
      unsigned long long acc = 0;
      for (long long g = 0; g < nseg; g++) {
        long long* v = p.segs + s * total + g * lines + line;
        const unsigned long long tot = (unsigned long long)*v;
        *v = (long long)acc;
        acc += tot;
      }
    }
}

// (3) each segment's inclusive prefix from its offset
__global__ void __launch_bounds__(kThreads) nd_scan_lines_write(KNDParams p, int d, const long long* in, long long* out) {
  const long long N = p.shape[d], step = p.inner[d];
  const long long total = (p.ncell / N) * ((N + kSeg - 1) / kSeg);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    long long base, i0, i1;
    seg_of(p, d, t, base, i0, i1);
    for (int s = 0; s < p.nstreams; s++) {
      unsigned long long acc = (unsigned long long)p.segs[s * total + t];
      for (long long i = i0; i < i1; i++) {
        acc += (unsigned long long)in[s * p.ncell + base + i * step];
        out[s * p.ncell + base + i * step] = (long long)acc;
      }
    }
  }
}

// Sliding sums along the contiguous dimension: one thread per cell.
__global__ void __launch_bounds__(kThreads) nd_pass_inner(KNDParams p, const long long* in, long long* out) {
  const int d = p.ndim - 1;
  const long long N = p.shape[d];
  const int h1 = p.h1[d], h2 = p.h2[d];
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < p.ncell; c += (long long)gridDim.x * blockDim.x) {
    const long long i = c % N, base = c - i;
    const long long a = max(0ll, i - h1), b = min(N - 1, i + h2);
    for (int s = 0; s < p.nstreams; s++) {
      const long long* src = in + s * p.ncell + base;
      unsigned long long acc = 0;
      for (long long j = a; j <= b; j++) acc += (unsigned long long)src[j];
      out[s * p.ncell + c] = (long long)acc;
    }
  }
}

// Inclusive prefix sums along the contiguous dimension: one warp per line,
// 32 cells at a time (warp scan plus the running carry).
__global__ void __launch_bounds__(kThreads) nd_scan_inner(KNDParams p, const long long* in, long long* out) {
  const int d = p.ndim - 1;
  const long long N = p.shape[d];
  const long long lines = p.ncell / N;
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long t = warp; t < lines; t += nwarps) {
    const long long base = t * N;
    for (int s = 0; s < p.nstreams; s++) {
      unsigned long long carry = 0;
      for (long long i0 = 0; i0 < N; i0 += 32) {
        const long long i = i0 + lane;
        unsigned long long v = i < N ? (unsigned long long)in[s * p.ncell + base + i] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned long long u = __shfl_up_sync(0xffffffffu, v, o);
          if (lane >= o) v += u;
        }
        v += carry;
        if (i < N) out[s * p.ncell + base + i] = (long long)v;
        carry = __shfl_sync(0xffffffffu, v, 31);
      }
    }
  }
}

// FP64 two-pass evaluation of the classical formula (Introduction) over the
// n-dimensional box [lo, hi] of the original grids, with the exact equality
// test for a constant channel.
static __device__ __noinline__ float nd_box_fp64(const KNDParams& p, const long long* lo, const long long* hi) {
  long long cur[KND_MAXDIM];
  double sx = 0.0, sy = 0.0, n = 0.0;
  float x0 = 0.0f, y0 = 0.0f;
  bool cx = true, cy = true;
  for (int pass = 0; pass < 2; pass++) {
    double mx = 0.0, my = 0.0, sxx = 0.0, syy = 0.0, sxy = 0.0;
    if (pass == 1) {
      if (cx || cy) return __int_as_float(0x7fc00000);
      mx = sx / n;
      my = sy / n;
    }
    for (int d = 0; d < p.ndim; d++) cur[d] = lo[d];
    while (true) {
      long long off = 0;
      for (int d = 0; d < p.ndim; d++) off += cur[d] * p.ipitch[d];
      float a, b;
      load_cell(p, off, a, b);
      if (pass == 0) {
        if (n == 0.0) {
          x0 = a;
          y0 = b;
        }
        cx = cx && a == x0;
        cy = cy && b == y0;
        sx += a;
        sy += b;
        n += 1.0;
      } else {
        const double u = (double)a - mx, v = (double)b - my;
        sxx += u * u;
        syy += v * v;
        sxy += u * v;
      }
      int d = p.ndim - 1;
      for (; d >= 0; d--) {
        if (cur[d] < hi[d]) {
          cur[d]++;
          break;
        }
        cur[d] = lo[d];
      }
      if (d < 0) break;
    }
    if (pass == 1) return (float)fmin(fmax(sxy / sqrt(sxx * syy), -1.0), 1.0);
  }
  return 0.0f;
}

// Window-local recomputation over the n-dimensional box [lo, hi]: the box's
// own range and map (fx_wide: up to 26 bits), exact 64-bit sums and Eq. 2 in
// 128-bit integers, certified as the grid map's windows are.  False when the
// certificate fails (the caller then takes nd_box_fp64).
static __device__ __noinline__ bool nd_box_exact(const KNDParams& p, const long long* lo, const long long* hi,
                                                 float* out) {
  long long cur[KND_MAXDIM];
  auto each = [&](auto&& fn) {
    for (int d = 0; d < p.ndim; d++) cur[d] = lo[d];
    while (true) {
      long long off = 0;
      for (int d = 0; d < p.ndim; d++) off += cur[d] * p.ipitch[d];
      float a, b;
      load_cell(p, off, a, b);
      fn(a, b);
      int d = p.ndim - 1;
      for (; d >= 0; d--) {
        if (cur[d] < hi[d]) {
          cur[d]++;
          break;
        }
        cur[d] = lo[d];
      }
      if (d < 0) break;
    }
  };
  float xlo = 3.0e38f, xhi = -3.0e38f, ylo = 3.0e38f, yhi = -3.0e38f;
  long long n = 0;
  each([&](float a, float b) {
    xlo = fminf(xlo, a); xhi = fmaxf(xhi, a); ylo = fminf(ylo, b); yhi = fmaxf(yhi, b);
    n++;
  });
  if (xlo == xhi || ylo == yhi) {  // a constant channel: zero variance, exactly
    *out = __int_as_float(0x7fc00000);
    return true;
  }
  const FxWide wx = fx_wide(xlo, xhi, n), wy = fx_wide(ylo, yhi, n);
  long long Sx = 0, Sy = 0, Sxx = 0, Syy = 0, Sxy = 0;
  bool okx = true, oky = true;
  each([&](float a, float b) {
    const long long X = fx_wide_quant(a, wx, okx), Y = fx_wide_quant(b, wy, oky);
    Sx += X; Sy += Y; Sxx += X * X; Syy += Y * Y; Sxy += X * Y;
  });
  const __int128 N = n;
  const __int128 vx = N * Sxx - (__int128)Sx * Sx;
  const __int128 vy = N * Syy - (__int128)Sy * Sy;
  const __int128 num = N * Sxy - (__int128)Sx * Sy;
  if (!fx_certified(i128_to_f32(vx), i128_to_f32(vy), (float)n, okx ? 0.0f : 0.5f, oky ? 0.0f : 0.5f)) return false;
  *out = fx_pearson128(num, vx, vy);
  return true;
}

__global__ void __launch_bounds__(kThreads) nd_finalize(KNDParams p, const long long* W) {
  const int* r = reinterpret_cast<const int*>(p.scratch);
  float rhox = 0.0f, rhoy = 0.0f;
  if (p.is_f32 && r[4]) {  // some value does not convert exactly
    rhox = map_of(p, 0).rho;
    rhoy = map_of(p, 1).rho;
  }
  uint32_t recomputed = 0;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < p.nout; o += (long long)gridDim.x * blockDim.x) {
    long long lo[KND_MAXDIM], hi[KND_MAXDIM];
    bool outside = false;
    long long rem = o, n = 1, centre_cell = 0;
    for (int d = p.ndim - 1; d >= 0; d--) {
      const long long j = rem % p.oshape[d];
      rem /= p.oshape[d];
      const long long c = j * p.stride[d];
      const long long a = c - p.h1[d], b = c + p.h2[d];
      outside = outside || a < 0 || b > p.shape[d] - 1;
      lo[d] = max(a, 0ll);
      hi[d] = min(b, p.shape[d] - 1);
      n *= hi[d] - lo[d] + 1;
      centre_cell += c * p.inner[d];
    }
    if (p.paper && outside) {
      p.out[o] = -2.0f;
      continue;
    }
    if (p.mask_only) {  // (uint16 grids hold no missing value)
      if (p.is_f32 && W[centre_cell] > 0) p.out[o] = -2.0f;
      continue;
    }
    long long S[6];
    if (!p.sat) {
      for (int s = 0; s < p.nstreams; s++) S[s] = W[s * p.ncell + centre_cell];
    } else {
      // inclusion-exclusion over the 2^ndim corners {lo - 1, hi} per dimension
      unsigned long long acc[6] = {0, 0, 0, 0, 0, 0};
      for (int m = 0; m < (1 << p.ndim); m++) {
        long long cell = 0;
        bool zero = false;
        int neg = 0;
        for (int d = 0; d < p.ndim; d++) {
          const bool take_lo = (m >> d) & 1;
          const long long i = take_lo ? lo[d] - 1 : hi[d];
          if (i < 0) zero = true;
          neg ^= take_lo ? 1 : 0;
          cell += i * p.inner[d];
        }
        if (zero) continue;
        for (int s = 0; s < p.nstreams; s++) {
          const unsigned long long v = (unsigned long long)W[s * p.ncell + cell];
          acc[s] = neg ? acc[s] - v : acc[s] + v;
        }
      }
      for (int s = 0; s < p.nstreams; s++) S[s] = (long long)acc[s];
    }
    if (p.sums) {
      long long* s5 = p.sums + 5 * o;
      for (int s = 0; s < 5; s++) s5[s] = S[s];
    }
    if (p.paper && S[5] > 0) {
      p.out[o] = -2.0f;
      continue;
    }
    const __int128 N = n;
    const __int128 vx = N * S[2] - (__int128)S[0] * S[0];
    const __int128 vy = N * S[3] - (__int128)S[1] * S[1];
    const __int128 num = N * S[4] - (__int128)S[0] * S[1];
    float c = fx_pearson128(num, vx, vy);  // a zero variance: 0 * rsqrt(0) = NaN
    if (p.is_f32 && !fx_certified(i128_to_f32(vx), i128_to_f32(vy), (float)n, rhox, rhoy)) {
      if (!nd_box_exact(p, lo, hi, &c)) c = nd_box_fp64(p, lo, hi);
      recomputed++;
    }
    p.out[o] = c;
  }
  if (recomputed) atomicAdd(p.status + ST_FALLBACK, recomputed);
}

// Mask-only form: -2 over the outputs whose index along d lies in [j0, j1)
// (one slab of windows that pass an edge of dimension d); inner = outputs
// per step of index d.
__global__ void __launch_bounds__(kThreads) nd_border_slab(KNDParams p, int d, long long j0, long long j1,
                                                           long long inner) {
  const long long width = j1 - j0, total = width * (p.nout / p.oshape[d]);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long in = t % inner, rest = t / inner;
    const long long j = j0 + rest % width, outer = rest / width;
    p.out[(outer * p.oshape[d] + j) * inner + in] = -2.0f;
  }
}

// Mask-only form, float32: -2 over the outputs whose window holds a missing
// cell (the summed count W at the window's centre), 32-bit index arithmetic
// (the plan keeps this form to outputs and cells below 2^31).
__global__ void __launch_bounds__(kThreads) nd_mask_apply(KNDParams p, const long long* W) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < (int)p.nout; o += gridDim.x * blockDim.x) {
    int rem = o;
    long long centre = 0;
    for (int d = p.ndim - 1; d >= 0; d--) {
      const int od = (int)p.oshape[d];
      const int j = rem % od;
      rem /= od;
      centre += (long long)j * p.stride[d] * p.inner[d];
    }
    if (W[centre] > 0) p.out[o] = -2.0f;
  }
}

}  // namespace

// The mask-only form's -2 over the windows that pass an edge: two slabs per
// dimension.
static cudaError_t knd_border(const KNDParams& p, int blocks, cudaStream_t st) {
  long long inner = 1;
  for (int d = p.ndim - 1; d >= 0; d--) {
    const long long O = p.oshape[d], s = p.stride[d], N = p.shape[d];
    // low side: j s - h1 < 0; high side: j s + h2 > N - 1
    const long long a = std::min(O, (p.h1[d] + s - 1) / s);
    const long long b = N - 1 - p.h2[d] < 0 ? 0 : std::min(O, (N - 1 - p.h2[d]) / s + 1);
    if (a > 0) nd_border_slab<<<blocks, kThreads, 0, st>>>(p, d, 0, a, inner);
    if (std::max(a, b) < O) nd_border_slab<<<blocks, kThreads, 0, st>>>(p, d, std::max(a, b), O, inner);
    inner *= O;
  }
  return cudaGetLastError();
}

cudaError_t knd_launch(const KNDParams& p, int sms, cudaStream_t st) {
  const int blocks = sms * 8;
  if (p.mask_only) {
    cudaError_t e = cudaSuccess;
    if (p.is_f32) {  // the missing-cell count, summed over each window, then applied
      nd_init<<<1, 1, 0, st>>>(p);
      nd_convert<<<blocks, kThreads, 0, st>>>(p);
      int cur = 0;
      for (int d = 0; d < p.ndim; d++) {
        if (d < p.ndim - 1)
          nd_pass_lines<<<blocks, kThreads, 0, st>>>(p, d, p.buf[cur], p.buf[cur ^ 1]);
        else
          nd_pass_inner<<<blocks, kThreads, 0, st>>>(p, p.buf[cur], p.buf[cur ^ 1]);
        cur ^= 1;
      }
      nd_mask_apply<<<blocks, kThreads, 0, st>>>(p, p.buf[cur]);
      e = cudaGetLastError();
    }
    return e == cudaSuccess ? knd_border(p, blocks, st) : e;
  }
  nd_init<<<1, 1, 0, st>>>(p);
  if (p.is_f32 && !p.mask_only) nd_range<<<blocks, kThreads, 0, st>>>(p);
  nd_convert<<<blocks, kThreads, 0, st>>>(p);
  int cur = 0;
  for (int d = 0; d < p.ndim; d++) {
    const long long* in = p.buf[cur];
    long long* out = p.buf[cur ^ 1];
    if (d < p.ndim - 1 && p.sat) {
      nd_scan_lines_totals<<<blocks, kThreads, 0, st>>>(p, d, in);
      nd_scan_lines_offsets<<<blocks, kThreads, 0, st>>>(p, d);
      nd_scan_lines_write<<<blocks, kThreads, 0, st>>>(p, d, in, out);
    } else if (d < p.ndim - 1)
      nd_pass_lines<<<blocks, kThreads, 0, st>>>(p, d, in, out);
    else if (p.sat)
      nd_scan_inner<<<blocks, kThreads, 0, st>>>(p, in, out);
    else
      nd_pass_inner<<<blocks, kThreads, 0, st>>>(p, in, out);
    cur ^= 1;
  }
  nd_finalize<<<blocks, kThreads, 0, st>>>(p, p.buf[cur]);
  return cudaGetLastError();
}

}  // namespace swc
