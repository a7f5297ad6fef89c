// k1d.cuh -- fused 1-D sliding-window correlation (uint16 or float32).
//
// The one-dimensional case of the optimized algorithm (Poyda & Zhizhin,
// Section 1: window sums in linear time like a rolling mean, then Eq. 2),
// for long windows (k up to 32*M1*stride + 1) on long series.
//
// One warp per work item = a chunk of 32*M1 consecutive outputs:
//  * The chunk's input span (its outputs' windows) is loaded into shared
//    memory with 1-D TMA boxes; cells before the start or past the end of the
//    series are zero filled and flagged off-grid.
//  * Values become exact integers: uint16 as they are, float32 through a
//    fixed-point map of the chunk (reference at the midpoint of the chunk's
//    range, power-of-two scale, |X| < 2^21), in place in shared memory.
//    Off-grid cells become 0.
//  * Lane j owns outputs j*M1 .. j*M1 + M1 - 1.  The span is cut into
//    segments of M1*stride cells, so lane j's first window starts at segment
//    j: it is q whole segments plus the first r cells of the next
//    (k = q*M1*stride + r).  Each lane sums its segments (totals of the five
//    streams, plus the sum of their first r cells); a warp scan of the
//    segment totals gives every lane its first window as a prefix difference.
//    All sums are modular integers (uint32 / uint64), hence exact.
//  * The lane then slides: window i+1 = window i + the stride cells that
//    enter - the stride cells that leave, and evaluates Eq. 2 exactly in int64
//    for each output (NaN for a zero variance), staged in shared memory and
//    stored coalesced.
#pragma once

#include "common.cuh"
#include "kparams.h"
#include "k1d_params.h"

namespace swc {

// Shared memory of one warp: X and Y as int32 (after conversion), the staged
// outputs, one mbarrier.
template <int M1>
struct Smem1D {
  static constexpr int L = 32 * M1;
};

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
  __device__ __forceinline__ void sub(int X, int Y) {
    x -= (uint32_t)X;
    y -= (uint32_t)Y;
    xx -= (uint64_t)((long long)X * X);
    yy -= (uint64_t)((long long)Y * Y);
    xy -= (uint64_t)((long long)X * Y);
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

// Eq. 2 from exact modular window sums (results fit in int64).
__device__ __forceinline__ float pearson_exact(const Sums5& s, uint64_t n) {
  const uint64_t s0 = (uint64_t)(long long)(int)s.x, s1 = (uint64_t)(long long)(int)s.y;
  const long long vx = (long long)(n * s.xx - s0 * s0);
  const long long vy = (long long)(n * s.yy - s1 * s1);
  const long long num = (long long)(n * s.xy - s0 * s1);
  // a zero variance makes num exactly 0, so 0 * rsqrt(0) = NaN
  return clamp1_nan(__ll2float_rn(num) * rsqrtf(__ll2float_rn(vx) * __ll2float_rn(vy)));
}

template <int M1>
__global__ void __launch_bounds__(32) k1d_kernel(const __grid_constant__ K1DParams p) {
  constexpr int L = 32 * M1;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // layout: X[span] int32, Y[span] int32, out[L] float, mbarrier
  int* X = reinterpret_cast<int*>(smem_raw);
  int* Y = X + p.span;
  float* so = reinterpret_cast<float*>(Y + p.span);
  uint64_t* bar = reinterpret_cast<uint64_t*>(so + L);
  const int lane = threadIdx.x;
  const int esz = p.is_f32 ? 4 : 2;
  const int align = 16 / esz;  // TMA start coordinate granularity
  if (lane == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncwarp();
  uint32_t phase = 0;
  const int seg = M1 * p.stride;

  for (long long item = blockIdx.x; item < p.n_items; item += gridDim.x) {
    const long long c0 = item * L;                        // first output of the chunk
    const long long e_first = c0 * p.stride - p.h1;       // first cell of its windows
    long long e0 = e_first >= 0 ? e_first / align * align : -((-e_first + align - 1) / align) * align;
    const int off = (int)(e_first - e0);                  // span offset of cell e_first
    // ---- load the span (raw values, zero filled off the series) into X/Y's bytes
    if (lane == 0) {
      fence_proxy_async_smem();
      if (p.gx != nullptr) {
        // (plain loads are done by the whole warp below)
      } else {
        mbar_arrive_expect_tx(bar, (uint32_t)(2 * p.nbox * 256 * esz));
        unsigned char* dx = reinterpret_cast<unsigned char*>(X);
        unsigned char* dy = reinterpret_cast<unsigned char*>(Y);
        for (int b = 0; b < p.nbox; b++) {
          tma_load_1d(dx + (size_t)b * 256 * esz, &p.tmx, (int)(e0 + 256ll * b), bar);
          tma_load_1d(dy + (size_t)b * 256 * esz, &p.tmy, (int)(e0 + 256ll * b), bar);
        }
      }
    }
    if (p.gx != nullptr) {
      for (int e = lane; e < p.nbox * 256; e += 32) {
        const long long g = e0 + e;
        const bool ok = g >= 0 && g < p.N;
        if (p.is_f32) {
          reinterpret_cast<float*>(X)[e] = ok ? __ldg((const float*)p.gx + g) : 0.0f;
          reinterpret_cast<float*>(Y)[e] = ok ? __ldg((const float*)p.gy + g) : 0.0f;
        } else {
          reinterpret_cast<uint16_t*>(X)[e] = ok ? __ldg((const uint16_t*)p.gx + g) : (uint16_t)0;
          reinterpret_cast<uint16_t*>(Y)[e] = ok ? __ldg((const uint16_t*)p.gy + g) : (uint16_t)0;
        }
      }
      __syncwarp();
    } else {
      if (!mbar_wait_bounded(bar, phase, p.status)) return;
      phase ^= 1u;
    }
    const int ncell = p.nbox * 256;
    // ---- convert to exact integers in place (read all, then write all)
    if (p.is_f32) {
      const float* fx = reinterpret_cast<const float*>(X);
      const float* fy = reinterpret_cast<const float*>(Y);
      float xlo = 3.0e38f, xhi = -3.0e38f, ylo = 3.0e38f, yhi = -3.0e38f;
      for (int e = lane; e < ncell; e += 32) {
        const long long g = e0 + e;
        if (g >= 0 && g < p.N) {
          xlo = fminf(xlo, fx[e]); xhi = fmaxf(xhi, fx[e]);
          ylo = fminf(ylo, fy[e]); yhi = fmaxf(yhi, fy[e]);
        }
      }
      xlo = warp_min(xlo); xhi = warp_max(xhi); ylo = warp_min(ylo); yhi = warp_max(yhi);
      float mx, sx, my, sy;
      {
        auto mk = [&](float lo, float hi, float& m, float& s) {
          if (!(lo <= hi)) lo = hi = 0.0f;
          m = lo + 0.5f * (hi - lo);
          const float A = fmaxf(hi - m, m - lo);
          int e = 0;
          if (A > 0.0f) {
            int ea;
            frexpf(A, &ea);
            e = min(max(p.qbits - ea, -126), 126);
          }
          s = __int_as_float((127 + e) << 23);
        };
        mk(xlo, xhi, mx, sx);
        mk(ylo, yhi, my, sy);
      }
      // in place: each lane converts its own cells (same index read then written)
      for (int e = lane; e < ncell; e += 32) {
        const long long g = e0 + e;
        const bool ok = g >= 0 && g < p.N;
        const float vx = fx[e], vy = fy[e];
        X[e] = ok ? __float_as_int(fmaf(vx - mx, sx, 12582912.0f)) - 0x4B400000 : 0;
        Y[e] = ok ? __float_as_int(fmaf(vy - my, sy, 12582912.0f)) - 0x4B400000 : 0;
      }
    } else {
      // uint16: widen in place, back to front so no cell is overwritten before it is read
      const uint16_t* ux = reinterpret_cast<const uint16_t*>(X);
      const uint16_t* uy = reinterpret_cast<const uint16_t*>(Y);
      for (int base = ((ncell - 1) / 32) * 32; base >= 0; base -= 32) {
        const int e = base + lane;
        int a = 0, b = 0;
        if (e < ncell) {
          a = ux[e];
          b = uy[e];
        }
        __syncwarp();
        if (e < ncell) {
          X[e] = a;
          Y[e] = b;
        }
        __syncwarp();
      }
    }
    __syncwarp();

    // ---- segment sums: segment g covers span cells [off + g*seg, off + (g+1)*seg)
    Sums5 T[2], R[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
      T[h].zero();
      R[h].zero();
      const int g = lane + 32 * h;
      if (g < p.nseg) {
        const int b = off + g * seg;
        for (int u = 0; u < seg; u++) {
          if (u == p.r) R[h] = T[h];
          const int e = b + u;
          if (e < ncell) T[h].add(X[e], Y[e]);
        }
        if (p.r >= seg) R[h] = T[h];
      }
    }
    // inclusive scan of the 64 segment totals (lanes, then the second half)
    Sums5 C0 = T[0], C1 = T[1];
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

    // ---- slide over the lane's outputs
    const long long j_base = c0 + (long long)lane * M1;
    int e_in = off + lane * seg + p.k;   // first cell to enter after the current window
    int e_out = off + lane * seg;        // first cell of the current window
    for (int t = 0; t < M1; t++) {
      const long long j = j_base + t;
      float cv = 0.0f;
      if (j < p.n_out) {
        const long long centre = j * p.stride;
        const long long lo = max(centre - p.h1, 0ll), hi = min(centre + p.h2, p.N - 1);
        cv = pearson_exact(W, (uint64_t)(hi - lo + 1));
      }
      so[lane * M1 + t] = cv;
      if (t + 1 < M1) {
        for (int u = 0; u < p.stride; u++) {
          const int ei = e_in + u, eo = e_out + u;
          if (ei < ncell) W.add(X[ei], Y[ei]);
          W.sub(X[eo], Y[eo]);
        }
        e_in += p.stride;
        e_out += p.stride;
      }
    }
    __syncwarp();
    // ---- coalesced store of the chunk's outputs
    const long long nvalid = min((long long)L, p.n_out - c0);
    for (int u = lane; u < nvalid; u += 32) p.out[c0 + u] = so[u];
    __syncwarp();
  }
}

}  // namespace swc
