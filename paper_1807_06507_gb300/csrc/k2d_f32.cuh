// k2d_f32.cuh -- fused 2-D sliding-window correlation for float32 grids.
//
// Same structure as the uint16 kernel (Poyda & Zhizhin, Section 1, steps 1-4
// fused; one warp per work item of 32*M centre columns x TJ output rows; a
// TMA-fed row ring; row pass as in-lane prefix differences of the entering-
// minus-leaving row, column pass as running sums), with one change of number
// system: float32 sums of squares cannot be evaluated to 1e-5 of the Pearson
// coefficient when a window's spread is small next to its offset, so each
// lane maps its values to integers and sums exactly.
//
//  * Pass 1 streams the item's rows through the ring once and takes, per
//    lane, the range [lo, hi] of x and of y over the lane's columns.
//  * Each value becomes X = round((x - m) s) with s = 2^e and m on the 2^-e
//    grid (fxmap.cuh), |X| < 2^q, q = 22 when the window has at most 511
//    cells and fewer above (n 2^q < 2^31 keeps the first-moment sums in
//    int32).  The affine map is the same for every window of the lane, so it
//    leaves Pearson's c unchanged; the rounding of each value is the only
//    error.
//  * Cells outside the grid must add nothing.  They are read as 0 (TMA zero
//    fill).  The lane's map has the subtract form (fxmap.cuh), and rows
//    outside the grid switch its reference to 0, which converts their zero
//    fill to exactly X = 0 (the missing leaving row of the first kh-1 rows
//    enters as 0 directly).  Columns outside the
//    grid, which only a few border lanes see, enter as the constant
//    G = X(0); since the sums are exact modular integers, step 4 subtracts
//    their known count times G, G^2 and Gx*Gy exactly.  (An off-grid column
//    is off-grid in the entering and the leaving row alike, so its entering-
//    minus-leaving differences are 0 or +-G and the products stay exact.)
//  * Pass 2 is the D-march with int32 first-moment and int64 second-moment
//    sums, all exact; step 4 evaluates n Sxy - Sx Sy etc. exactly in int64 and
//    rounds once to float32 per factor.  A zero variance gives NaN exactly.
//  * Each window's result is certified (fxmap.cuh): with rho the lane's
//    rounding bound, |dc| <= rho n (1/sqrt(vx) + 1/sqrt(vy)) + 7e-7.  The
//    common case passes a one-comparison-per-channel test (lanes of integer
//    data on a grid step of at most 1 convert exactly, rho = 0: nothing to
//    test).  A window that does not pass flags its lane.  After the item,
//    each flagged lane determines whether its values convert exactly (then
//    its results stand); the others march again through the ring with a
//    finer map of the same range (up to 26 bits, 64-bit sums, Eq. 2 in
//    128-bit integers), which certifies the windows of ordinary float data
//    whose spread is small next to the lane's range.  Plain plans list that
//    second tier as tasks of a few output rows for a second launch, which
//    spreads them over every SM (a few listed items no longer hold up the
//    whole grid); batched plans and host-run bands run it inside the item.
//    Windows that still fail (a value orders of magnitude above its
//    neighbours in the lane's columns) are recomputed from their own cells
//    by the whole warp at once.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "fxmap.cuh"
#include "kparams.h"

namespace swc {

template <int M, int KW>
struct Geo2DF {
  static constexpr int W1 = (KW - 1) / 2;
  static constexpr int W2 = KW / 2;
  static constexpr int HALO = (W1 <= 8 && W2 <= 8) ? 8 : 16;
  static constexpr int RW = 32 * M + 2 * HALO;     // floats per row and channel
  static constexpr int RWS = (RW + 31) / 32 * 32;  // ring row stride (128-byte rows)
  static constexpr int NMAIN = RW / 256;
  static constexpr int TAIL = RW - 256 * NMAIN;
  static constexpr int OFF = HALO - W1;
  static constexpr int CH0 = OFF / 4;              // first float4 of the lane
  static constexpr int E0 = OFF % 4;
  static constexpr int NCOL = M + KW - 1;
  static constexpr int NCH = (E0 + NCOL + 3) / 4;  // float4 chunks per lane, row and channel
  static_assert(TAIL % 4 == 0 && NMAIN >= 1, "row span cannot be split into TMA boxes");
  static_assert(M % 4 == 0, "lane base must be 16-byte aligned");
};

struct Ring2DF {
  float* rx;      // entering rows [NR][RWS]
  float* ry;
  float* lx;      // leaving rows (pass 2) [NR][RWS]
  float* ly;
  uint64_t* bar;  // [NR]
  int NR;
  int PF;
  uint32_t* pend; // windows the lane re-march could not certify: (row - j0) << 8 | lane << 3 | column
  int* npend;     //   (at most kPend2D per item; the count may run past it)
};

constexpr int kPend2D = 512;

struct FixScene2D {  // the fields of a scene the fix-up reads (passed by value)
  const float* gx;
  const float* gy;
  long long in_pitch;
  int H, W, h1, h2, kh, kw, sx, sy;
};

// Whether every in-grid value of a lane's item (rows [r0, r1), the lane's
// NCOL columns from c0, those with index in [e_lo, e_hi) inside the grid)
// converts without rounding under the lane's maps.  Integer data on a grid
// step of at most 1 passes a cheap first test (x - m and (x - m) s are then
// exact); otherwise every value is tested (fx_on_grid).  Each row's loads
// are independent, so they are in flight together.
template <int NCOL>
static __device__ __noinline__ bool lane_exact_2d(const float* gx, const float* gy, long long pitch, int r0, int r1,
                                                  int c0, int e_lo, int e_hi, FxMap qx, FxMap qy) {
  for (int pass = (qx.s >= 1.0f && qy.s >= 1.0f) ? 0 : 1; pass < 2; pass++) {
    bool ok = true;
    for (int r = r0; r < r1 && ok; r++) {  // (a lane stops at its first value off the grid)
      const long long o = (long long)r * pitch + c0;
      float vx[NCOL], vy[NCOL];
#pragma unroll
      for (int e = 0; e < NCOL; e++) {
        vx[e] = (e >= e_lo && e < e_hi) ? gx[o + e] : 0.0f;
        vy[e] = (e >= e_lo && e < e_hi) ? gy[o + e] : 0.0f;
      }
#pragma unroll
      for (int e = 0; e < NCOL; e++) {
        if (pass == 0)
          ok = ok && vx[e] == rintf(vx[e]) && vy[e] == rintf(vy[e]);
        else if (e >= e_lo && e < e_hi)
          ok = ok && fx_on_grid(vx[e], qx) && fx_on_grid(vy[e], qy);
      }
    }
    if (ok) return true;
  }
  return false;
}

// Recompute the window of centre (jr sy, cc) from its cells, the whole warp
// together (fx_box_warp), and store it over the earlier result.
static __device__ __noinline__ void fix_window_warp_2d(const FixScene2D& sc, float* out, long long out_pitch, int jr,
                                                       int cc) {
  // (arguments are the same in every lane)
  if (cc >= sc.W || (sc.sx != 1 && cc % sc.sx != 0)) return;
  const int rc = jr * sc.sy, w1 = (sc.kw - 1) / 2, w2 = sc.kw / 2;
  FxBox b;
  b.gx = sc.gx;
  b.gy = sc.gy;
  b.pz = 0;
  b.py = sc.in_pitch;
  b.z0 = b.z1 = 0;
  b.y0 = max(rc - sc.h1, 0);
  b.y1 = min(rc + sc.h2, sc.H - 1);
  b.x0 = max(cc - w1, 0);
  b.x1 = min(cc + w2, sc.W - 1);
  const float c = fx_box_warp(b, nullptr);
  if ((threadIdx.x & 31) == 0) out[(long long)jr * out_pitch + (sc.sx == 1 ? cc : cc / sc.sx)] = c;
}

// The windows the second tier could not certify (the whole warp calls it):
// each listed window, then every window of a lane whose list overflowed, is
// recomputed by the whole warp from its own cells (fx_box_warp).
template <int M>
static __device__ __noinline__ void fix_listed_2d(FixScene2D sc, float* out, long long out_pitch, const uint32_t* pend,
                                                  int npend, bool ovf, int cl, int j0, int j1, uint32_t* status) {
  const int lane = threadIdx.x & 31;
  const int n = min(npend, kPend2D);
  for (int i = 0; i < n; i++) {
    const uint32_t e = pend[i];
    const int l = (int)(e >> 3) & 31;
    fix_window_warp_2d(sc, out, out_pitch, j0 + (int)(e >> 8), cl - M * lane + M * l + (int)(e & 7));
  }
  uint32_t om = __ballot_sync(0xffffffffu, ovf);
  while (om) {
    const int l = __ffs(om) - 1;
    om &= om - 1;
    for (int jr = j0; jr < j1; jr++)
      for (int c = 0; c < M; c++) fix_window_warp_2d(sc, out, out_pitch, jr, cl - M * lane + M * l + c);
  }
  if (lane == 0 && n > 0) atomicAdd(status + ST_FALLBACK, (uint32_t)n);
}

// The second tier's placement, a compile-time choice so that each kernel
// instance holds the registers of the passes it runs.
enum : int {
  TIER_IN_PLACE = 0,  // the whole item, second tier inside it (batched plans, host-run bands)
  TIER_LIST = 1,      // the item's first tier; its second tier listed as tasks
  TIER_TASK = 2       // one listed task: the second tier only
};

// Output rows [j0, j1) of column strip `strip` (TIER_TASK: the lanes in
// task_lanes, with the ranges of their item at range slot task_slot).
template <int M, int KW, bool TMA, int TIER>
__device__ __forceinline__ bool process_rows_2d_f32(const Scene2D& sc, int strip, int j0, int j1, uint32_t task_lanes,
                                                    int task_slot, const Ring2DF& rg, uint32_t& seq,
                                                    uint32_t* status) {
  using G = Geo2DF<M, KW>;
  const int lane = threadIdx.x & 31;
  constexpr bool task = TIER == TIER_TASK;
  const int t0 = j0 * sc.sy - sc.h1;
  const int nrows = (j1 - 1 - j0) * sc.sy + sc.kh;
  const int cstrip = strip * 32 * M;
  const int xs = cstrip - G::HALO;
  const uint32_t NR = (uint32_t)rg.NR;
  const int PF = rg.PF;

  // row `row` into slot s (entering part) and, when lrow is on the item's
  // leaving side (pass 2, i >= kh), row lrow into the leaving part
  auto issue = [&](uint32_t s, int row, bool with_leave, int lrow) {
    if (!TMA) {
      auto copy_row = [&](float* dx, float* dy, int r) {
        const bool row_ok = r >= 0 && r < sc.H;
        const float* gx = (const float*)sc.gx + (long long)(row_ok ? r : 0) * sc.in_pitch;
        const float* gy = (const float*)sc.gy + (long long)(row_ok ? r : 0) * sc.in_pitch;
        for (int e = lane; e < G::RW; e += 32) {
          const int col = xs + e;
          const bool ok = row_ok && col >= 0 && col < sc.W;
          dx[e] = ok ? __ldg(gx + col) : 0.0f;
          dy[e] = ok ? __ldg(gy + col) : 0.0f;
        }
      };
      copy_row(rg.rx + (size_t)s * G::RWS, rg.ry + (size_t)s * G::RWS, row);
      if (with_leave) copy_row(rg.lx + (size_t)s * G::RWS, rg.ly + (size_t)s * G::RWS, lrow);
      return;
    }
    uint64_t* b = rg.bar + s;
    mbar_arrive_expect_tx(b, (with_leave ? 2u : 1u) * 2u * G::RW * 4u);
    auto row_boxes = [&](float* dx, float* dy, int r) {
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
    if (with_leave) row_boxes(rg.lx + (size_t)s * G::RWS, rg.ly + (size_t)s * G::RWS, lrow);
  };

  // One streaming pass over the item's rows through the ring: issue ahead,
  // wait, hand the slot to body(i, slot), keep the ring bookkeeping.
  auto stream_rows = [&](bool leaving, auto&& body) -> bool {
    uint32_t s = seq % NR, lap = (seq / NR) & 1u, sp = (s + (uint32_t)PF) % NR;
    {
      const int npre = min(PF, nrows);
      if (!TMA || lane == 0) {
        if (TMA) fence_proxy_async_smem();
        uint32_t si = s;
        for (int i = 0; i < npre; i++) {
          issue(si, t0 + i, leaving && i >= sc.kh, t0 + i - sc.kh);
          si = (si + 1 == NR) ? 0u : si + 1;
        }
      }
    }
    for (int i = 0; i < nrows; i++) {
      __syncwarp();
      if (i + PF < nrows && (!TMA || lane == 0)) {
        if (TMA) fence_proxy_async_smem();
        issue(sp, t0 + i + PF, leaving && i + PF >= sc.kh, t0 + i + PF - sc.kh);
      }
      sp = (sp + 1 == NR) ? 0u : sp + 1;
      if (!TMA) {
        __syncwarp();
      } else if (!mbar_wait_bounded(rg.bar + s, lap, status)) {
        uint32_t sk = s, lk = lap;
        for (int k = i + 1; k <= min(i + PF, nrows - 1); k++) {
          sk = (sk + 1 == NR) ? 0u : sk + 1;
          if (sk == 0u) lk ^= 1u;
          mbar_wait_bounded(rg.bar + sk, lk, status);
        }
        return false;
      }
      // the first kh rows of an item have no leaving row (compile-time phase)
      if (i < sc.kh)
        body(i, s, std::false_type{});
      else
        body(i, s, std::true_type{});
      s = (s + 1 == NR) ? 0u : s + 1;
      if (s == 0u) lap ^= 1u;
    }
    seq += (uint32_t)nrows;
    __syncwarp();
    return true;
  };

  const int cl = cstrip + M * lane;
  auto lane_ptr = [&](const float* ring, uint32_t slot) {
    return ring + (size_t)slot * G::RWS + M * lane + G::CH0 * 4;
  };

  // ---- pass 1: value range of the lane's columns over the item's rows
  float xlo = 3.0e38f, xhi = -3.0e38f, ylo = 3.0e38f, yhi = -3.0e38f;
  bool allint = true;  // every value an integer (then, with s >= 1, every value converts exactly)
  // in-grid columns of the lane: e in [e_lo, e_hi)
  const int e_lo = max(0, G::W1 - cl), e_hi = min(G::NCOL, sc.W - (cl - G::W1));
  if constexpr (task) {  // a task re-marches with the ranges its item measured
    const float4 r = sc.redo_ranges[32 * task_slot + lane];
    xlo = r.x; xhi = r.y; ylo = r.z; yhi = r.w;
  } else if (!stream_rows(false, [&](int i, uint32_t s, auto) {
        if (t0 + i < 0 || t0 + i >= sc.H) return;
        const float* px = lane_ptr(rg.rx, s);
        const float* py = lane_ptr(rg.ry, s);
#pragma unroll
        for (int h = 0; h < G::NCH; h++) {
          const float4 a = *reinterpret_cast<const float4*>(px + 4 * h);
          const float4 b = *reinterpret_cast<const float4*>(py + 4 * h);
          const float va[4] = {a.x, a.y, a.z, a.w}, vb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
          for (int u = 0; u < 4; u++) {
            const int e = 4 * h + u - G::E0;
            if (e >= 0 && e < G::NCOL && e >= e_lo && e < e_hi) {
              xlo = fminf(xlo, va[u]);
              xhi = fmaxf(xhi, va[u]);
              ylo = fminf(ylo, vb[u]);
              yhi = fmaxf(yhi, vb[u]);
              // |v| + 1.5*2^23 rounds |v| < 2^22 to an integer (larger |v| may
              // fail the test; they are then checked in full if needed)
              allint = allint && (fabsf(va[u]) + kFxMagic) - kFxMagic == fabsf(va[u]) &&
                       (fabsf(vb[u]) + kFxMagic) - kFxMagic == fabsf(vb[u]);
            }
          }
        }
      }))
    return false;

  // subtract form (C = 1.5*2^23): rows outside the grid take the reference 0,
  // which converts their zero fill to X = 0
  const FxMap qx = fx_make(xlo, xhi, sc.qbits, false), qy = fx_make(ylo, yhi, sc.qbits, false);
  float mxe = qx.msub, mye = qy.msub, mxl = qx.msub, myl = qy.msub;  // per-row references
  const bool lane_border = (cl - G::W1 < 0) || (cl + M - 1 + G::W2 > sc.W - 1);
  const int Gx = fx_quant(0.0f, qx), Gy = fx_quant(0.0f, qy);  // value of an off-grid column
  // quick certificate: vx >= (rho n / 4.5e-6)^2 with n the interior count
  // (border windows have fewer cells, so the test is conservative there)
  // lane exactness: -1 not yet known, 0 no, 1 yes (integers on a grid step of
  // at most 1: x - m and (x - m) s are exact)
  const int exact_state = (allint && qx.s >= 1.0f && qy.s >= 1.0f) ? 1 : -1;
  bool need = false;  // a window of the lane failed its quick certificate test
  float Kx, Ky;  // quick certificate thresholds, fixed for the item
  {
    const float nmax = (float)(sc.kh * KW);
    const float k0 = 4.9432e10f * nmax * nmax;  // (1 / 4.5e-6)^2 * 1.001
    Kx = exact_state == 1 ? 0.0f : k0 * qx.rho * qx.rho;
    Ky = exact_state == 1 ? 0.0f : k0 * qy.rho * qy.rho;
  }

  const bool fast_cols = sc.sx == 1 && sc.vec_store;
  uint32_t n_c[M];
#pragma unroll
  for (int c = 0; c < M; c++) {
    const int cc = cl + c;
    n_c[c] = (uint32_t)(sc.kh * max(min(cc + G::W2, sc.W - 1) - max(cc - G::W1, 0) + 1, 1));
  }

  // exact modular sums (wrapping unsigned arithmetic)
  uint32_t V0[M], V1[M];
  uint64_t V2[M], V3[M], V4[M];
#pragma unroll
  for (int c = 0; c < M; c++) {
    V0[c] = 0u; V1[c] = 0u; V2[c] = 0ull; V3[c] = 0ull; V4[c] = 0ull;
  }
  int until_out = sc.kh - 1;
  int jr = j0;
  const uint32_t seq0 = seq;

  // ---- pass 2: the D-march on fixed-point values
  bool ok = true;
  if constexpr (!task) ok = stream_rows(true, [&](int i, uint32_t s, auto leave_tag) {
    constexpr bool has_leave = decltype(leave_tag)::value;
    const int te = t0 + i, tl = te - sc.kh;
    const bool e_ok = te >= 0 && te < sc.H;
    const bool l_ok = has_leave && tl >= 0 && tl < sc.H;
    mxe = e_ok ? qx.msub : 0.0f;
    mye = e_ok ? qy.msub : 0.0f;
    mxl = l_ok ? qx.msub : 0.0f;
    myl = l_ok ? qy.msub : 0.0f;
    const float* pxe = lane_ptr(rg.rx, s);
    const float* pye = lane_ptr(rg.ry, s);
    const float* pxl = lane_ptr(rg.lx, s);
    const float* pyl = lane_ptr(rg.ly, s);
    uint32_t P0 = 0u, P1 = 0u;
    uint64_t P2 = 0ull, P3 = 0ull, P4 = 0ull;
    uint32_t Ps0[M], Ps1[M];
    uint64_t Ps2[M], Ps3[M], Ps4[M];
#pragma unroll
    for (int h = 0; h < G::NCH; h++) {
      const float4 a = *reinterpret_cast<const float4*>(pxe + 4 * h);
      const float4 b = *reinterpret_cast<const float4*>(pye + 4 * h);
      float4 al = make_float4(0.f, 0.f, 0.f, 0.f), bl = al;
      if constexpr (has_leave) {
        al = *reinterpret_cast<const float4*>(pxl + 4 * h);
        bl = *reinterpret_cast<const float4*>(pyl + 4 * h);
      }
      const float xa[4] = {a.x, a.y, a.z, a.w}, ya[4] = {b.x, b.y, b.z, b.w};
      const float xla[4] = {al.x, al.y, al.z, al.w}, yla[4] = {bl.x, bl.y, bl.z, bl.w};
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int e = 4 * h + u - G::E0;
        if (e < 0 || e >= G::NCOL) continue;
        const int Xe = fx_quant_sub(xa[u], mxe, qx.s), Xl = has_leave ? fx_quant_sub(xla[u], mxl, qx.s) : 0;
        const int Ye = fx_quant_sub(ya[u], mye, qy.s), Yl = has_leave ? fx_quant_sub(yla[u], myl, qy.s) : 0;
        const int D = (int)((uint32_t)Xe - (uint32_t)Xl), S = (int)((uint32_t)Xe + (uint32_t)Xl);
        const int Dy = (int)((uint32_t)Ye - (uint32_t)Yl), Sy = (int)((uint32_t)Ye + (uint32_t)Yl);
        P0 += (uint32_t)D;
        P1 += (uint32_t)Dy;
        P2 += (uint64_t)((long long)D * S);
        P3 += (uint64_t)((long long)Dy * Sy);
        P4 += (uint64_t)((long long)D * Ye) + (uint64_t)((long long)Xl * Dy);
        if (e >= KW - 1) {
          const int c = e - (KW - 1);
          V0[c] += P0 - (c >= 1 ? Ps0[c - 1] : 0u);
          V1[c] += P1 - (c >= 1 ? Ps1[c - 1] : 0u);
          V2[c] += P2 - (c >= 1 ? Ps2[c - 1] : 0ull);
          V3[c] += P3 - (c >= 1 ? Ps3[c - 1] : 0ull);
          V4[c] += P4 - (c >= 1 ? Ps4[c - 1] : 0ull);
        }
        if (e <= M - 2) {
          Ps0[e] = P0; Ps1[e] = P1; Ps2[e] = P2; Ps3[e] = P3; Ps4[e] = P4;
        }
      }
    }

    if (until_out == 0) {
      until_out = sc.sy;
      const int rc = jr * sc.sy;
      const int cnt_r = min(rc + sc.h2, sc.H - 1) - max(rc - sc.h1, 0) + 1;
      float* orow = sc.out + (long long)jr * sc.out_pitch;
      if (lane_border) {
        // remove the off-grid columns' constant contribution (exact, modular)
#pragma unroll
        for (int c = 0; c < M; c++) {
          const uint32_t n_oob = (uint32_t)(cnt_r * (KW - (int)(n_c[c] / (uint32_t)sc.kh)));
          V0[c] -= n_oob * (uint32_t)Gx;
          V1[c] -= n_oob * (uint32_t)Gy;
          V2[c] -= (uint64_t)n_oob * (uint64_t)((long long)Gx * Gx);
          V3[c] -= (uint64_t)n_oob * (uint64_t)((long long)Gy * Gy);
          V4[c] -= (uint64_t)n_oob * (uint64_t)((long long)Gx * Gy);
        }
      }
      float res[M];
      uint32_t fail = 0;  // windows whose quick certificate test failed
#pragma unroll
      for (int c = 0; c < M; c++) {
        const uint64_t n = cnt_r == sc.kh ? (uint64_t)n_c[c] : (uint64_t)(n_c[c] / sc.kh * cnt_r);
        // exact in 64-bit modular arithmetic; the results are below 2^63
        const uint64_t s0 = (uint64_t)(long long)(int)V0[c], s1 = (uint64_t)(long long)(int)V1[c];
        const long long vx = (long long)(n * V2[c] - s0 * s0);
        const long long vy = (long long)(n * V3[c] - s1 * s1);
        const long long num = (long long)(n * V4[c] - s0 * s1);
        const float fvx = i64_to_f32(vx), fvy = i64_to_f32(vy);
        // a zero variance makes num exactly 0, so 0 * rsqrt(0) = NaN
        res[c] = clamp1_nan(i64_to_f32(num) * rsqrtf(fvx * fvy));
        // windows past the grid's last column have no certificate to pass
        // (strided plans drop non-output columns in the fix-up)
        fail |= (fvx >= Kx && fvy >= Ky) || cl + c >= sc.W ? 0u : (1u << c);
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
      // rare: a window the item map cannot certify (the lane's windows are
      // recomputed after the item, unless the lane converts exactly)
      if (fail != 0u && exact_state != 1) need = true;
      if (lane_border) {
        // restore the running sums for the next rows
#pragma unroll
        for (int c = 0; c < M; c++) {
          const uint32_t n_oob = (uint32_t)(cnt_r * (KW - (int)(n_c[c] / (uint32_t)sc.kh)));
          V0[c] += n_oob * (uint32_t)Gx;
          V1[c] += n_oob * (uint32_t)Gy;
          V2[c] += (uint64_t)n_oob * (uint64_t)((long long)Gx * Gx);
          V3[c] += (uint64_t)n_oob * (uint64_t)((long long)Gy * Gy);
          V4[c] += (uint64_t)n_oob * (uint64_t)((long long)Gx * Gy);
        }
      }
      jr++;
    }
    until_out--;
  });
  (void)seq0;
  if (!ok) return false;
  __syncwarp();

  // ---- pass 3 (second tier): lanes whose item map left a window
  // uncertified and whose values do not all convert exactly march the item
  // again through the ring with a finer map of the same range, fx_wide (up to
  // 26 bits, 64-bit sums; values on the grid exact, others within 1/2), and
  // evaluate Eq. 2 in 128-bit integers.  Cells outside the grid are absent
  // (X = 0, not counted).  Two passes of M/2 windows each (the 64-bit running
  // sums of all M windows would not fit the registers).  Every window of the
  // lane is rewritten; those that still fail are listed for the warp.
  bool redo = false;
  if constexpr (task) {
    // a task's lanes were found inexact by the launch that listed them; a
    // channel constant over the task's cells leaves exact NaN results
    redo = ((task_lanes >> lane) & 1u) && xlo < xhi && ylo < yhi;
  } else if (__any_sync(0xffffffffu, need)) {
    const bool exact = exact_state == 1 ||
                       (need && exact_state < 0 &&
                        lane_exact_2d<G::NCOL>((const float*)sc.gx, (const float*)sc.gy, sc.in_pitch, max(t0, 0),
                                               min(t0 + nrows, sc.H), cl - G::W1, e_lo, e_hi, qx, qy));
    // a channel constant over the lane's cells makes every window's variance
    // exactly zero: the item map's results (NaN) stand
    redo = need && !exact && xlo < xhi && ylo < yhi;
    if constexpr (TIER == TIER_LIST) {
      // list the item's second tier as tasks of redo_rows output rows for
      // the next launch, which spreads them over every SM (the plan sizes
      // the list for every item's tasks, so it cannot fill; if it did, the
      // plan's status reports it)
      const uint32_t lanes = __ballot_sync(0xffffffffu, redo);
      if (lanes) {
        const int nt = (j1 - j0 + sc.redo_rows - 1) / sc.redo_rows;
        int k = 0;
        if (lane == 0) k = atomicAdd(sc.redo_count, nt);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k + nt <= sc.redo_cap) {
          const int slot = (j0 / sc.TJ) * sc.n_strips + strip;  // the item's index (plain plans: one launch)
          sc.redo_ranges[32 * slot + lane] = make_float4(xlo, xhi, ylo, yhi);
          for (int t = lane; t < nt; t += 32)
            sc.redo_tasks[k + t] =
                RedoTask2D{strip, j0 + t * sc.redo_rows, min(j0 + (t + 1) * sc.redo_rows, j1), lanes, slot, {0, 0, 0}};
        } else if (lane == 0) {
          atomicOr(status + ST_ERROR, ERRBIT_BAD_ARG);
        }
      }
      redo = false;
    }
  }
  if constexpr (TIER != TIER_LIST) if (__any_sync(0xffffffffu, redo)) {
    if (lane == 0) *rg.npend = 0;
    __syncwarp();
    const long long nmax = (long long)sc.kh * KW;
    const FxWide wx = fx_wide(xlo, xhi, nmax), wy = fx_wide(ylo, yhi, nmax);
    bool ongx = true, ongy = true;  // every value read so far lies on its channel's grid
    bool ovf = false;
    uint32_t count = 0;
    // Windows up to 15 columns wide march all M windows in one pass: a row's
    // first-moment contribution to a window, |sum of D| < 15 * 2^27.02, fits
    // in 32 bits, which leaves registers for the 64-bit running sums.  Wider
    // windows take two passes of M/2 windows.
    constexpr int PARTS = KW <= 15 ? 1 : 2;
    using T1 = std::conditional_t<PARTS == 1, uint32_t, unsigned long long>;
    auto redo_pass = [&](auto half_tag) -> bool {
      constexpr int HALF = decltype(half_tag)::value;
      constexpr int MH = M / PARTS, NC = MH + KW - 1, EB = HALF * MH;  // lane columns [EB, EB + NC)
      constexpr int HB = (G::E0 + EB) / 4, HE = (G::E0 + EB + NC - 1) / 4 + 1;
      unsigned long long V[MH][5];
#pragma unroll
      for (int c = 0; c < MH; c++)
#pragma unroll
        for (int t = 0; t < 5; t++) V[c][t] = 0ull;
      int until_out = sc.kh - 1;
      int jr = j0;
      return stream_rows(true, [&](int i, uint32_t s, auto leave_tag) {
        constexpr bool has_leave = decltype(leave_tag)::value;
        if (redo) {
          const int te = t0 + i, tl = te - sc.kh;
          const bool e_ok = te >= 0 && te < sc.H;
          const bool l_ok = has_leave && tl >= 0 && tl < sc.H;
          const float* pxe = lane_ptr(rg.rx, s);
          const float* pye = lane_ptr(rg.ry, s);
          const float* pxl = lane_ptr(rg.lx, s);
          const float* pyl = lane_ptr(rg.ly, s);
          T1 P01[2] = {0u, 0u};
          unsigned long long P[5] = {0ull, 0ull, 0ull, 0ull, 0ull};  // (entries 2-4 used)
          T1 Ps01[MH > 1 ? MH - 1 : 1][2];
          unsigned long long Ps[MH > 1 ? MH - 1 : 1][5];              // (entries 2-4 used)
          auto ext = [](T1 v) -> unsigned long long {  // a row contribution, sign-extended
            if constexpr (sizeof(T1) == 4)
              return (unsigned long long)(long long)(int)v;
            else
              return v;
          };
#pragma unroll
          for (int h = HB; h < HE; h++) {
            const float4 a = *reinterpret_cast<const float4*>(pxe + 4 * h);
            const float4 b = *reinterpret_cast<const float4*>(pye + 4 * h);
            float4 al = make_float4(0.f, 0.f, 0.f, 0.f), bl = al;
            if constexpr (has_leave) {
              al = *reinterpret_cast<const float4*>(pxl + 4 * h);
              bl = *reinterpret_cast<const float4*>(pyl + 4 * h);
            }
            const float xa[4] = {a.x, a.y, a.z, a.w}, ya[4] = {b.x, b.y, b.z, b.w};
            const float xla[4] = {al.x, al.y, al.z, al.w}, yla[4] = {bl.x, bl.y, bl.z, bl.w};
#pragma unroll
            for (int u = 0; u < 4; u++) {
              const int e = 4 * h + u - G::E0;
              if (e < EB || e >= EB + NC) continue;
              const bool cok = e >= e_lo && e < e_hi;
              long long Xe = 0, Ye = 0, Xl = 0, Yl = 0;
              if (e_ok && cok) {
                Xe = fx_wide_quant(xa[u], wx, ongx);
                Ye = fx_wide_quant(ya[u], wy, ongy);
              }
              if (l_ok && cok) {
                Xl = fx_wide_quant(xla[u], wx, ongx);
                Yl = fx_wide_quant(yla[u], wy, ongy);
              }
              // |X| < 2^26 (1 + 2^-6) + 1: differences, sums and their
              // products fit 32 x 32 -> 64-bit multiplies
              const int D = (int)(Xe - Xl), S = (int)(Xe + Xl), Dy = (int)(Ye - Yl), Sy = (int)(Ye + Yl);
              P01[0] += (T1)(long long)D;
              P01[1] += (T1)(long long)Dy;
              P[2] += (unsigned long long)((long long)D * S);
              P[3] += (unsigned long long)((long long)Dy * Sy);
              P[4] += (unsigned long long)((long long)D * (int)Ye + (long long)(int)Xl * Dy);
              const int j = e - EB;
              if (j >= KW - 1) {
                const int c = j - (KW - 1);
                V[c][0] += ext(P01[0] - (c >= 1 ? Ps01[c - 1][0] : (T1)0u));
                V[c][1] += ext(P01[1] - (c >= 1 ? Ps01[c - 1][1] : (T1)0u));
#pragma unroll
                for (int t = 2; t < 5; t++) V[c][t] += P[t] - (c >= 1 ? Ps[c - 1][t] : 0ull);
              }
              if (j <= MH - 2) {
                Ps01[j][0] = P01[0];
                Ps01[j][1] = P01[1];
#pragma unroll
                for (int t = 2; t < 5; t++) Ps[j][t] = P[t];
              }
            }
          }
        }
        if (until_out == 0) {
          until_out = sc.sy;
          if (redo) {
            const int rc = jr * sc.sy;
            const long long cnt_r = min(rc + sc.h2, sc.H - 1) - max(rc - sc.h1, 0) + 1;
            float* orow = sc.out + (long long)jr * sc.out_pitch;
#pragma unroll
            for (int c = 0; c < MH; c++) {
              const int cc = cl + EB + c;
              if (cc < sc.W && (sc.sx == 1 || cc % sc.sx == 0)) {
                const long long n = cnt_r * (min(cc + G::W2, sc.W - 1) - max(cc - G::W1, 0) + 1);
                const long long s0 = (long long)V[c][0], s1 = (long long)V[c][1];
                const __int128 vx = (__int128)n * (long long)V[c][2] - (__int128)s0 * s0;
                const __int128 vy = (__int128)n * (long long)V[c][3] - (__int128)s1 * s1;
                const __int128 num = (__int128)n * (long long)V[c][4] - (__int128)s0 * s1;
                float r = __int_as_float(0x7fc00000);
                if (fx_certified(i128_to_f32(vx), i128_to_f32(vy), (float)n, ongx ? 0.0f : 0.5f,
                                 ongy ? 0.0f : 0.5f)) {
                  r = fx_pearson128(num, vx, vy);
                } else {
                  const int k = atomicAdd(rg.npend, 1);
                  if (k < kPend2D)
                    rg.pend[k] = ((uint32_t)(jr - j0) << 8) | ((uint32_t)lane << 3) | (uint32_t)(EB + c);
                  else
                    ovf = true;
                }
                orow[sc.sx == 1 ? cc : cc / sc.sx] = r;
                count++;
              }
            }
          }
          jr++;
        }
        until_out--;
      });
    };
    if (!redo_pass(std::integral_constant<int, 0>{})) return false;
    if constexpr (PARTS == 2)
      if (!redo_pass(std::integral_constant<int, 1>{})) return false;
    if (count) atomicAdd(status + ST_FALLBACK, count);
    __syncwarp();
    const FixScene2D fs{(const float*)sc.gx, (const float*)sc.gy, sc.in_pitch, sc.H, sc.W, sc.h1, sc.h2, sc.kh, KW,
                        sc.sx, sc.sy};
    fix_listed_2d<M>(fs, sc.out, sc.out_pitch, rg.pend, *rg.npend, ovf, cl, j0, j1, status);
  }
  return true;
}

template <int M, int KW, bool TMA>
__device__ __forceinline__ bool process_item_2d_f32(const Scene2D& sc, int strip, int rb, const Ring2DF& rg,
                                                    uint32_t& seq, uint32_t* status) {
  const int j0 = rb * sc.TJ;
  return process_rows_2d_f32<M, KW, TMA, TIER_IN_PLACE>(sc, strip, j0, min(j0 + sc.TJ, sc.OH), 0u, 0, rg, seq, status);
}

}  // namespace swc
