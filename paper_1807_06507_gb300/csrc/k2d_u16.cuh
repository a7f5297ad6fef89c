// k2d_u16.cuh -- fused 2-D sliding-window correlation for uint16 grids.
//
// Steps 1-4 of the optimized algorithm (Poyda & Zhizhin, Section 1) in one
// pass over HBM, for one work item = (column strip of 32*M centre columns)
// x (TJ output rows), processed by one warp:
//
//  * Rows stream into shared-memory rings by TMA (one 2-D box row per
//    input row, zero fill outside the grid = the clipped border): the row
//    entering the column window and, separately, the row leaving it (read
//    again from L2 kh rows later), so the ring depth does not grow with kh.
//  * Step 1 (products) is formed on the fly from the entering row e and the
//    leaving row l = e - kh of each column: d = x_e - x_l, s = x_e + x_l,
//    x_e^2 - x_l^2 = d*s, x_e y_e - x_l y_l = d_x y_e + x_l d_y.
//  * Step 2 (row pass, window kw): in-lane prefix sums of those differences
//    over the lane's M + kw - 1 columns; a window is a prefix difference.
//  * Step 3 (column pass, window kh): register-resident running sums V, one
//    per output column, updated by the row-pass difference of each new row.
//  * Step 4: Pearson from the sums (Eq. 2), stored as float32.
//
// All sums are kept modulo 2^32, which is exact for sum x and sum y.  Step 4
// below needs T_x, T_y < 2^32 and |U| < 2^31.  A lane certifies all windows
// of an output row at once from the range R of the values it has loaded in
// the item (T <= n (R^2/4 + 5), |U| <= sqrt(T_x T_y)); a row that fails is
// evaluated per window: certified by M_w * Sx < 2^32 (M_w the running
// maximum, so sum x^2 <= M_w Sx) and T_x T_y < 2^62, else recomputed exactly
// in int64 from global memory and counted.
//
// Finalize, exact up to the last float32 roundings: with a = an integer near
// the window mean and r = Sx - n a,
//     T_x = sum (x - a)^2 = Sxx - a (Sx + r),   n Sxx - Sx^2 = n T_x - r^2,
// and the same for y and for the cross term U = Sxy - b Sx - a s,
// n Sxy - Sx Sy = n U - r s.  T_x, T_y < 2^32 (certified) and |U| < 2^31
// (checked through T_x T_y < 2^62), so they are exact in 32-bit arithmetic;
// each Pearson factor is then one fused multiply-add in float32.  A zero
// variance is detected exactly.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "kparams.h"

namespace swc {

template <int M, int KW>
struct Geo2D {
  static constexpr int W1 = (KW - 1) / 2;         // window columns left of the centre
  static constexpr int W2 = KW / 2;               // ... right of the centre
  static constexpr int HALO = (W1 <= 8 && W2 <= 8) ? 8 : 16;
  static constexpr int RW = 32 * M + 2 * HALO;    // elements loaded per row and channel
  // TMA writes must start on 128-byte boundaries: ring rows are padded to a
  // multiple of 64 elements and a row is loaded as NMAIN boxes of 256
  // elements plus one TAIL box (both 128-byte aligned in shared memory).
  static constexpr int RWS = (RW + 63) / 64 * 64; // ring row stride (elements)
  static constexpr int NMAIN = RW / 256;
  static constexpr int TAIL = RW - 256 * NMAIN;
  static constexpr int OFF = HALO - W1;           // first needed element, from the lane base
  static constexpr int CH0 = OFF / 8;             // first 16-byte chunk, from the lane base
  static constexpr int E0 = OFF % 8;              // element offset inside that chunk
  static constexpr int NCOL = M + KW - 1;         // columns each lane sums
  static constexpr int NCH = (E0 + NCOL + 7) / 8; // 16-byte chunks per lane, row and channel
  static constexpr int NWORD = 4 * NCH;
  static_assert(TAIL % 8 == 0 && NMAIN >= 1, "row span cannot be split into TMA boxes");
  static_assert(M % 8 == 0, "lane base must be 16-byte aligned");
  static_assert(KW >= 1 && KW <= 31, "kw out of range");
};

struct Ring2D {
  uint16_t* rx;  // entering rows, [NR][RWS]
  uint16_t* ry;
  uint16_t* lx;  // leaving rows, [NR][RWS]
  uint16_t* ly;
  uint64_t* bar; // [NR]: one phase per (entering, leaving) pair
  int NR;        // = PF + 1
  int PF;
};

__device__ __forceinline__ uint32_t get16(const uint32_t* w, int idx) {
  const uint32_t v = w[idx >> 1];
  return (idx & 1) ? (v >> 16) : (v & 0xFFFFu);
}

// Exact per-window recomputation (rare path): int64 sums over the window's
// in-grid cells read from global memory, Pearson in fp64.
static __device__ __noinline__ float exact_window_u16(const Scene2D& sc, int rc, int cc, int kw, int n, long long* out5) {
  const int w1 = (kw - 1) / 2, w2 = kw / 2;
  const uint16_t* gx = (const uint16_t*)sc.gx;
  const uint16_t* gy = (const uint16_t*)sc.gy;
  long long sx = 0, sy = 0, sxx = 0, syy = 0, sxy = 0;
  for (int r = max(rc - sc.h1, 0); r <= min(rc + sc.h2, sc.H - 1); r++)
    for (int c = max(cc - w1, 0); c <= min(cc + w2, sc.W - 1); c++) {
      const long long a = gx[(long long)r * sc.in_pitch + c], b = gy[(long long)r * sc.in_pitch + c];
      sx += a;
      sy += b;
      sxx += a * a;
      syy += b * b;
      sxy += a * b;
    }
  if (out5) {
    out5[0] = sx; out5[1] = sy; out5[2] = sxx; out5[3] = syy; out5[4] = sxy;
  }
  const long long vx = (long long)n * sxx - sx * sx;
  const long long vy = (long long)n * syy - sy * sy;
  const long long num = (long long)n * sxy - sx * sy;
  if (vx == 0 || vy == 0) return __int_as_float(0x7fc00000);
  double cv = (double)num / sqrt((double)vx * (double)vy);
  cv = fmin(fmax(cv, -1.0), 1.0);
  return (float)cv;
}

// Plain-load row loader (for row pitches that are not a multiple of 16 bytes,
// which TMA cannot describe): the warp copies one input row span into a ring
// slot, writing zeros outside the grid exactly as the TMA zero fill does.
template <int RW>
__device__ __forceinline__ void ldg_row_u16(uint16_t* dst, const uint16_t* src, long long pitch, int row, int xs,
                                            int H, int W, int lane) {
  const bool row_ok = row >= 0 && row < H;
  const uint16_t* r = src + (long long)(row_ok ? row : 0) * pitch;
  for (int e = lane; e < RW; e += 32) {
    const int col = xs + e;
    dst[e] = (row_ok && col >= 0 && col < W) ? __ldg(r + col) : (uint16_t)0;
  }
}

// Step 4 for one output from its exact modular window sums (see the file
// header).  Valid when Sxx, Syy < 2^32 (certified by the caller) and
// T_x T_y < 2^62, i.e. |U| < 2^31: the caller checks tt = T_x T_y.
__device__ __forceinline__ float pearson_u16(uint32_t Sx, uint32_t Sy, uint32_t Sxx, uint32_t Syy, uint32_t Sxy,
                                             uint32_t n, float fn, uint32_t a, uint32_t b, float& tt) {
  const int r = (int)(Sx - n * a), s = (int)(Sy - n * b);
  const uint32_t Tx = Sxx - a * (Sx + (uint32_t)r);
  const uint32_t Ty = Syy - b * (Sy + (uint32_t)s);
  const int U = (int)(Sxy - b * Sx - a * (uint32_t)s);
  const float fr = __int2float_rn(r), fs = __int2float_rn(s);
  const float fTx = __uint2float_rn(Tx), fTy = __uint2float_rn(Ty);
  tt = fTx * fTy;
  const float vx = fmaf(fn, fTx, -fr * fr);
  const float vy = fmaf(fn, fTy, -fs * fs);
  const float num = fmaf(fn, __int2float_rn(U), -fr * fs);
  // A zero variance makes num exactly 0 (all values of one channel equal:
  // n Sxy - Sx Sy = 0 in integers, and every term above is exact), so
  // num * rsqrt(0) = 0 * inf = NaN, which the clamp keeps.
  return clamp1_nan(num * rsqrtf(vx * vy));
}

// Certificate: with every value of the window <= Mv, the second moment is
// <= Mv * S; Mv * S < 2^32 for both channels makes Sxx and Syy exact.
__device__ __forceinline__ bool certified(uint32_t Mx, uint32_t Sx, uint32_t My, uint32_t Sy) {
  return (__umulhi(Mx, Sx) == 0u) && (__umulhi(My, Sy) == 0u);
}

// |U| <= sqrt(T_x T_y) < 2^31 when T_x T_y < 2^62 (float product, margin kept).
constexpr float TT_LIMIT = 4.0e18f;

// Process one work item.  Returns false if a bounded wait gave up (the
// caller must then exit; in-flight copies have been drained).
// WIDE = false: the certified 32-bit engine described above.  WIDE = true
// (large windows, n = kh*kw > 64, where second moments routinely exceed
// 2^32): the second-moment sums are exact 64-bit integers and step 4 is
// evaluated exactly in int64, with no certificate.
template <int M, int KW, bool TMA, bool WIDE = false>
__device__ __forceinline__ bool process_item_2d_u16(const Scene2D& sc, int strip, int rb, const Ring2D& rg,
                                                    uint32_t& seq, uint32_t* status) {
  using G = Geo2D<M, KW>;
  const int lane = threadIdx.x & 31;
  const int j0 = rb * sc.TJ;
  const int j1 = min(j0 + sc.TJ, sc.OH);
  const int t0 = j0 * sc.sy - sc.h1;
  const int nrows = (j1 - 1 - j0) * sc.sy + sc.kh;
  const int cstrip = strip * 32 * M;
  const int xs = cstrip - G::HALO;
  const uint32_t NR = (uint32_t)rg.NR;
  const int PF = rg.PF;

  // entering row i (and, once i >= kh, leaving row i - kh) into slot s
  auto issue = [&](uint32_t s, int i) {
    const int row = t0 + i;
    const bool lv = i >= sc.kh;
    if (!TMA) {
      ldg_row_u16<G::RW>(rg.rx + (size_t)s * G::RWS, (const uint16_t*)sc.gx, sc.in_pitch, row, xs, sc.H, sc.W,
                         lane);
      ldg_row_u16<G::RW>(rg.ry + (size_t)s * G::RWS, (const uint16_t*)sc.gy, sc.in_pitch, row, xs, sc.H, sc.W,
                         lane);
      if (lv) {
        ldg_row_u16<G::RW>(rg.lx + (size_t)s * G::RWS, (const uint16_t*)sc.gx, sc.in_pitch, row - sc.kh, xs, sc.H,
                           sc.W, lane);
        ldg_row_u16<G::RW>(rg.ly + (size_t)s * G::RWS, (const uint16_t*)sc.gy, sc.in_pitch, row - sc.kh, xs, sc.H,
                           sc.W, lane);
      }
      return;
    }
    uint64_t* b = rg.bar + s;
    mbar_arrive_expect_tx(b, (lv ? 2u : 1u) * 2u * G::RW * 2u);
    if (sc.test_stall && strip == 0 && rb == 0 && i == 0) return;  // the failure-path test hook
    auto row_boxes = [&](uint16_t* dx, uint16_t* dy, int r) {
#pragma unroll
      for (int q = 0; q < G::NMAIN; q++) {
        tma_load_2d(dx + q * 256, sc.tmx, xs + q * 256, r, b);
        tma_load_2d(dy + q * 256, sc.tmy, xs + q * 256, r, b);
      }
      if (G::TAIL > 0) {
        tma_load_2d(dx + G::NMAIN * 256, sc.tmx_t, xs + G::NMAIN * 256, r, b);
        tma_load_2d(dy + G::NMAIN * 256, sc.tmy_t, xs + G::NMAIN * 256, r, b);
      }
    };
    row_boxes(rg.rx + (size_t)s * G::RWS, rg.ry + (size_t)s * G::RWS, row);
    if (lv) row_boxes(rg.lx + (size_t)s * G::RWS, rg.ly + (size_t)s * G::RWS, row - sc.kh);
  };

  // Ring bookkeeping without divisions in the row loop: slot of row i, its
  // mbarrier phase, and the prefetch slot.
  uint32_t s = seq % NR;
  uint32_t lap = (seq / NR) & 1u;
  uint32_t sp = (s + (uint32_t)PF) % NR;
  {
    const int npre = min(PF, nrows);
    if (!TMA || lane == 0) {
      if (TMA) fence_proxy_async_smem();
      uint32_t si = s;
      for (int i = 0; i < npre; i++) {
        issue(si, i);
        si = (si + 1 == NR) ? 0u : si + 1;
      }
    }
  }

  const int cl = cstrip + M * lane;
  const bool fast_cols = sc.sx == 1 && sc.sums == nullptr && sc.vec_store;
  // Window size n, its float and floor(2^32 / n) (mean estimate) for each of
  // the lane's columns on interior rows; border columns have clipped counts.
  uint32_t n_c[M], inv_c[M];
  float fn_c[M];
#pragma unroll
  for (int c = 0; c < M; c++) {
    const int cc = cl + c;
    const int cnt_c = max(min(cc + G::W2, sc.W - 1) - max(cc - G::W1, 0) + 1, 1);
    n_c[c] = (uint32_t)(sc.kh * cnt_c);
    fn_c[c] = (float)n_c[c];
    inv_c[c] = n_c[c] == (uint32_t)(sc.kh * KW) ? sc.inv_n : __float2uint_rz(4294967296.0f * __frcp_rn(fn_c[c]));
  }

  using Acc = typename std::conditional<WIDE, uint64_t, uint32_t>::type;
  uint32_t V[M][2];  // sum x, sum y
  Acc VQ[M][3];      // sum x^2, sum y^2, sum xy
#pragma unroll
  for (int c = 0; c < M; c++) {
    V[c][0] = V[c][1] = 0u;
    VQ[c][0] = VQ[c][1] = VQ[c][2] = (Acc)0;
  }
  uint32_t mx2 = 0u, my2 = 0u;             // running maxima (two uint16 per word)
  uint32_t mn2 = 0xFFFFFFFFu, mny2 = 0xFFFFFFFFu;  // running minima
  int until_out = sc.kh - 1;  // rows until the next output row is complete
  int jr = j0;

  // One row step; LEAVE is false for the first kh rows of the item, which
  // have no leaving row (their row pass works on the entering row alone).
  auto step = [&](int i, auto leave_tag) -> bool {
    constexpr bool LEAVE = decltype(leave_tag)::value;
    __syncwarp();
    if (i + PF < nrows && (!TMA || lane == 0)) {
      if (TMA) fence_proxy_async_smem();
      issue(sp, i + PF);
    }
    sp = (sp + 1 == NR) ? 0u : sp + 1;
    if (!TMA) {
      __syncwarp();
    } else if (!mbar_wait_bounded(rg.bar + s, lap, status)) {
      // drain every copy still in flight into this CTA's ring, then give up
      uint32_t sk = s, lk = lap;
      for (int k = i + 1; k <= min(i + PF, nrows - 1); k++) {
        sk = (sk + 1 == NR) ? 0u : sk + 1;
        if (sk == 0u) lk ^= 1u;
        mbar_wait_bounded(rg.bar + sk, lk, status);
      }
      return false;
    }
    constexpr bool has_leave = LEAVE;

    uint32_t we[G::NWORD], wl[G::NWORD], ye[G::NWORD], yl[G::NWORD];
    {
      const uint16_t* pe = rg.rx + (size_t)s * G::RWS + M * lane + G::CH0 * 8;
      const uint16_t* qe = rg.ry + (size_t)s * G::RWS + M * lane + G::CH0 * 8;
#pragma unroll
      for (int h = 0; h < G::NCH; h++) {
        const uint4 a = *reinterpret_cast<const uint4*>(pe + 8 * h);
        const uint4 b = *reinterpret_cast<const uint4*>(qe + 8 * h);
        we[4 * h] = a.x; we[4 * h + 1] = a.y; we[4 * h + 2] = a.z; we[4 * h + 3] = a.w;
        ye[4 * h] = b.x; ye[4 * h + 1] = b.y; ye[4 * h + 2] = b.z; ye[4 * h + 3] = b.w;
      }
      if constexpr (has_leave) {
        const uint16_t* pl = rg.lx + (size_t)s * G::RWS + M * lane + G::CH0 * 8;
        const uint16_t* ql = rg.ly + (size_t)s * G::RWS + M * lane + G::CH0 * 8;
#pragma unroll
        for (int h = 0; h < G::NCH; h++) {
          const uint4 a = *reinterpret_cast<const uint4*>(pl + 8 * h);
          const uint4 b = *reinterpret_cast<const uint4*>(ql + 8 * h);
          wl[4 * h] = a.x; wl[4 * h + 1] = a.y; wl[4 * h + 2] = a.z; wl[4 * h + 3] = a.w;
          yl[4 * h] = b.x; yl[4 * h + 1] = b.y; yl[4 * h + 2] = b.z; yl[4 * h + 3] = b.w;
        }
      } else {
#pragma unroll
        for (int w = 0; w < G::NWORD; w++) { wl[w] = 0u; yl[w] = 0u; }
      }
    }
#pragma unroll
    for (int w = 0; w + 1 < G::NWORD; w += 2) {
      mx2 = __vimax3_u16x2(mx2, we[w], we[w + 1]);
      my2 = __vimax3_u16x2(my2, ye[w], ye[w + 1]);
      if (!WIDE) {
        mn2 = __vimin3_u16x2(mn2, we[w], we[w + 1]);
        mny2 = __vimin3_u16x2(mny2, ye[w], ye[w + 1]);
      }
    }

    // Row pass on the entering-minus-leaving differences, then the running
    // column sums.
    uint32_t P[2] = {0u, 0u};
    Acc PQ[3] = {(Acc)0, (Acc)0, (Acc)0};
    uint32_t Pst[M][2];  // prefix after column e, kept for output e + 1
    Acc PQst[M][3];
#pragma unroll
    for (int e = 0; e < G::NCOL; e++) {
      const uint32_t xe = get16(we, G::E0 + e), xl = get16(wl, G::E0 + e);
      const uint32_t yv = get16(ye, G::E0 + e), ylv = get16(yl, G::E0 + e);
      const uint32_t dx = xe - xl, sxs = xe + xl;
      const uint32_t dy = yv - ylv, sys = yv + ylv;
      P[0] += dx;
      P[1] += dy;
      if (WIDE) {
        PQ[0] += (Acc)((long long)(int)dx * (int)sxs);
        PQ[1] += (Acc)((long long)(int)dy * (int)sys);
        PQ[2] += (Acc)((long long)(int)dx * (int)yv + (long long)(int)xl * (int)dy);
      } else {
        PQ[0] += (Acc)(dx * sxs);
        PQ[1] += (Acc)(dy * sys);
        PQ[2] += (Acc)(dx * yv + xl * dy);
      }
      if (e >= KW - 1) {
        const int c = e - (KW - 1);
#pragma unroll
        for (int k = 0; k < 2; k++) V[c][k] += P[k] - (c >= 1 ? Pst[c - 1][k] : 0u);
#pragma unroll
        for (int k = 0; k < 3; k++) VQ[c][k] += PQ[k] - (c >= 1 ? PQst[c - 1][k] : (Acc)0);
      }
      if (e <= M - 2) {
#pragma unroll
        for (int k = 0; k < 2; k++) Pst[e][k] = P[k];
#pragma unroll
        for (int k = 0; k < 3; k++) PQst[e][k] = PQ[k];
      }
    }

    s = (s + 1 == NR) ? 0u : s + 1;
    if (s == 0u) lap ^= 1u;

    // Step 4 for the output row whose window is now complete.
    if (WIDE && until_out == 0) {
      until_out = sc.sy;
      const int rc = jr * sc.sy;
      const int cnt_r = min(rc + sc.h2, sc.H - 1) - max(rc - sc.h1, 0) + 1;
      float* orow = sc.out + (long long)jr * sc.out_pitch;
      float res[M];
#pragma unroll
      for (int c = 0; c < M; c++) {
        const uint64_t n = cnt_r == sc.kh ? (uint64_t)n_c[c] : (uint64_t)(n_c[c] / (uint32_t)sc.kh * (uint32_t)cnt_r);
        const uint64_t s0 = V[c][0], s1 = V[c][1];
        // exact in 64-bit arithmetic; a zero variance makes num 0 and c NaN
        const long long vx = (long long)(n * (uint64_t)VQ[c][0] - s0 * s0);
        const long long vy = (long long)(n * (uint64_t)VQ[c][1] - s1 * s1);
        const long long num = (long long)(n * (uint64_t)VQ[c][2] - s0 * s1);
        res[c] = clamp1_nan(i64_to_f32(num) * rsqrtf(i64_to_f32(vx) * i64_to_f32(vy)));
        const int cc = cl + c;
        if (sc.sums && cc < sc.W && (sc.sx == 1 || cc % sc.sx == 0)) {
          long long* s5 = sc.sums + 5ll * ((long long)jr * sc.OW + (sc.sx == 1 ? cc : cc / sc.sx));
          s5[0] = (long long)s0; s5[1] = (long long)s1;
          s5[2] = (long long)VQ[c][0]; s5[3] = (long long)VQ[c][1]; s5[4] = (long long)VQ[c][2];
        }
      }
      if (fast_cols && cl + M <= sc.W) {
#pragma unroll
        for (int c = 0; c < M; c += 4) stg128(orow + cl + c, res[c], res[c + 1], res[c + 2], res[c + 3]);
      } else {
#pragma unroll
        for (int c = 0; c < M; c++) {
          const int cc = cl + c;
          if (cc < sc.W && (sc.sx == 1 || cc % sc.sx == 0)) orow[sc.sx == 1 ? cc : cc / sc.sx] = res[c];
        }
      }
      jr++;
    } else if (until_out == 0) {
      until_out = sc.sy;
      const int rc = jr * sc.sy;
      const uint32_t Mx = max(mx2 & 0xFFFFu, mx2 >> 16), My = max(my2 & 0xFFFFu, my2 >> 16);
      const bool row_interior = (rc - sc.h1 >= 0) && (rc + sc.h2 <= sc.H - 1);
      float* orow = sc.out + (long long)jr * sc.out_pitch;
      // One certificate for every window of the lane's row: with R the range
      // of the values the lane has loaded in this item (its windows' cells
      // among them), T = sum (x - a)^2 <= n (R^2 / 4 + 5) (Popoviciu's bound
      // plus (mean - a)^2 < 5) and |U| <= sqrt(T_x T_y); T_x, T_y < 2^32 and
      // T_x T_y < 2^62 make the 32-bit evaluation exact.
      const float n_max = (float)(sc.kh * KW);
      const uint32_t rng_x = Mx - min(mn2 & 0xFFFFu, mn2 >> 16), rng_y = My - min(mny2 & 0xFFFFu, mny2 >> 16);
      const float bx = n_max * fmaf(0.25f * (float)rng_x, (float)rng_x, 5.0f);
      const float by = n_max * fmaf(0.25f * (float)rng_y, (float)rng_y, 5.0f);
      const bool row_cert = bx < 4.2e9f && by < 4.2e9f && bx * by < 4.5e18f;
      const bool fast = fast_cols && row_interior && __all_sync(0xffffffffu, row_cert);
      if (fast) {
        float res[M];
#pragma unroll
        for (int c = 0; c < M; c++) {
          float tt;
          res[c] = pearson_u16(V[c][0], V[c][1], (uint32_t)VQ[c][0], (uint32_t)VQ[c][1], (uint32_t)VQ[c][2], n_c[c], fn_c[c],
                               __umulhi(V[c][0], inv_c[c]), __umulhi(V[c][1], inv_c[c]), tt);
        }
        if (cl + M <= sc.W) {
#pragma unroll
          for (int c = 0; c < M; c += 4) stg128(orow + cl + c, res[c], res[c + 1], res[c + 2], res[c + 3]);
        } else {
#pragma unroll
          for (int c = 0; c < M; c++)
            if (cl + c < sc.W) orow[cl + c] = res[c];
        }
      }
      if (!fast) {
        // border rows or lanes, strided columns, debug sums, or a row whose
        // certificate needs the per-window test: per-output n and checks
        const int cnt_r = min(rc + sc.h2, sc.H - 1) - max(rc - sc.h1, 0) + 1;
#pragma unroll
        for (int c = 0; c < M; c++) {
          const int cc = cl + c;
          if (cc < sc.W && (sc.sx == 1 || (cc % sc.sx) == 0)) {
            const int cnt_c = min(cc + G::W2, sc.W - 1) - max(cc - G::W1, 0) + 1;
            const uint32_t n = (uint32_t)(cnt_r * cnt_c);
            const float fn = (float)n;
            const float rn = 1.0f / fn;
            const uint32_t a = (uint32_t)((float)V[c][0] * rn), b = (uint32_t)((float)V[c][1] * rn);
            const int jc = sc.sx == 1 ? cc : cc / sc.sx;
            long long* s5 = sc.sums ? sc.sums + 5ll * ((long long)jr * sc.OW + jc) : nullptr;
            float cv = 0.0f, tt = TT_LIMIT;
            if (certified(Mx, V[c][0], My, V[c][1]))
              cv = pearson_u16(V[c][0], V[c][1], (uint32_t)VQ[c][0], (uint32_t)VQ[c][1], (uint32_t)VQ[c][2], n, fn, a, b,
                               tt);
            if (tt < TT_LIMIT) {
              if (s5) {
                s5[0] = V[c][0]; s5[1] = V[c][1];
                s5[2] = (uint32_t)VQ[c][0]; s5[3] = (uint32_t)VQ[c][1]; s5[4] = (uint32_t)VQ[c][2];
              }
            } else {
              // rare: sums that may not be exact in 32 bits, recomputed exactly
              cv = exact_window_u16(sc, rc, cc, KW, (int)n, s5);
              atomicAdd(status + ST_FALLBACK, 1u);
            }
            orow[jc] = cv;
          }
        }
      }
      jr++;
    }
    until_out--;
    return true;
  };
  {
    const int nw = min(sc.kh, nrows);
    for (int i = 0; i < nw; i++)
      if (!step(i, std::false_type{})) return false;
    for (int i = nw; i < nrows; i++)
      if (!step(i, std::true_type{})) return false;
  }
  seq += (uint32_t)nrows;
  return true;
}

// One warp per CTA, persistent over the plan's work items: 16 resident CTAs
// per SM for the 32-bit engine; the 64-bit engine is held to 12 up to 17
// columns, 8 above.
template <int M, int KW, bool TMA, bool WIDE>
__global__ void __launch_bounds__(32, WIDE ? (KW <= 17 ? 12 : 8) : (KW <= 3 ? 16 : 12)) k2d_u16_kernel(const __grid_constant__ K2DParams p) {
  using G = Geo2D<M, KW>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Ring2D rg;
  rg.NR = p.NR;
  rg.PF = p.PF;
  rg.rx = reinterpret_cast<uint16_t*>(smem_raw);
  rg.ry = rg.rx + (size_t)p.NR * G::RWS;
  rg.lx = rg.ry + (size_t)p.NR * G::RWS;
  rg.ly = rg.lx + (size_t)p.NR * G::RWS;
  rg.bar = reinterpret_cast<uint64_t*>(rg.ly + (size_t)p.NR * G::RWS);
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
  for (int item = blockIdx.x; item < p.n_items; item += gridDim.x) {
    const int rbi = item / sc.n_strips;
    const int strip = item - rbi * sc.n_strips;
    const int rb = p.rb0 + rbi;
    if (!process_item_2d_u16<M, KW, TMA, WIDE>(sc, strip, rb, rg, seq, p.status)) return;
  }
}

}  // namespace swc
