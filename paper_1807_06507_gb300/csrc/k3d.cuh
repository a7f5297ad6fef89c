// k3d.cuh -- fused 3-D sliding-window correlation (uint16 or float32).
//
// The n-dimensional generalisation of the optimized algorithm (Poyda &
// Zhizhin, Section 1: one sliding-sum pass per dimension; parallel scheme of
// Section 2 extended to the third dimension), fused into one kernel.
//
// A CTA of 128 threads owns a footprint of TY output rows x TX output
// columns and marches along z over a block of TZ output planes:
//  * Each z-step brings the entering plane (z + kz/2) and the leaving plane
//    (z - (kz-1)/2 - 1) of the footprint's input rectangle into shared memory
//    with 3-D TMA boxes (zero fill off the volume); the leaving plane comes
//    back from L2, where it was read kz steps earlier.
//  * Values become exact integers: uint16 as they are (off-volume cells 0);
//    float32 through one fixed-point map per work item (fxmap.cuh), taken in
//    a first pass over its planes, with |X| < 2^q, q <= 22 chosen so that the
//    int64 evaluation of Eq. 2 cannot overflow (n 2^q < 2^31.5 * 1.0156, the
//    map's 1/64 margin) and a plane's window sums fit in int32.  The window's
//    sum of X is kept modulo 2^32: it is exact as an int32 whenever
//    n Sxx < 2^62 (Cauchy-Schwarz: |Sx| <= sqrt(n Sxx) < 2^31); a window
//    beyond that is treated as one whose certificate fails.  Off-volume cells
//    convert to X = 0 through a zero scale and the plain rounding constant
//    1.5*2^23, switched per plane, column and row.
//  * Vertical pass: one thread per input column forms, for every row of the
//    rectangle, the five entering-minus-leaving streams (x, y, x^2, y^2, xy
//    differences), their running prefix down the column, and the window sums
//    of ky rows as prefix differences (snapshots kept in registers); the
//    results go to a structure-of-arrays buffer.
//  * Horizontal pass: each lane takes 4 output columns of 2 output rows, sums
//    kx columns of that buffer as prefix differences, and adds the result to
//    its running 3-D sums (registers), which are therefore the sums over the
//    kz x ky x kx window of the current output plane.
//  * Step 4 (Eq. 2) exactly in int64 once the plane's window is complete.
// All sums are modular integers (uint32 / uint64), hence exact.
//  * float32 certificate (fxmap.cuh), evaluated in step 4 from the two
//    rsqrt factors of c: z = rho n (1/sqrt(vx) + 1/sqrt(vy)) <= 8.99e-6.  An
//    item in which some window fails asks the whole CTA, after its z-march,
//    whether its values convert exactly (rho = 0); if not, it is listed for
//    a second launch of the same kernel in its wide form, which marches the
//    listed items again with a map of up to 26 bits (64-bit first moments,
//    Eq. 2 in 128-bit integers) and rewrites their windows; the windows that
//    still fail are recomputed from their own cells, one warp per window.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "fxmap.cuh"
#include "kparams.h"

namespace swc {

struct K3DParams {
  CUtensorMap tmx;  // 3-D maps: dims {W, H, Z}, box {BXW, TY + ky - 1, 1}
  CUtensorMap tmy;
  int Z, H, W;
  int kz, hz1, hz2;
  int sz, sy, sx;
  int OZ, OY, OX;
  int TZ;            // output planes per work item
  int nzb, nyb, nxb;
  int n_items;
  int is_f32;
  int qbits;
  long long opz, opy;  // output pitches (elements) of a plane and of a row
  float* out;
  uint32_t* status;
  int use_tma;         // 0: plain loads (pitches TMA cannot describe)
  const void* gx;
  const void* gy;
  long long ipy, ipz;  // input pitches (elements) of a row and of a plane
  int unit_stride;     // sz = sy = sx = 1
  int vec_store;       // output rows 16-byte aligned (unit strides)
  long long* sums;     // optional (uint16): 5 int64 per output in C order, Sx Sy Sxx Syy Sxy
  // float32: items whose windows the 22-bit item map left uncertified (the
  // first kernel appends them; the wide kernel re-marches them)
  int* redo_count;
  int* redo_items;
};

constexpr int K3_THREADS = 128;

template <int TY, int TX, int KY, int KX>
struct Geo3D {
  static constexpr int H1 = (KY - 1) / 2, H2 = KY / 2;
  static constexpr int W1 = (KX - 1) / 2, W2 = KX / 2;
  static constexpr int TYI = TY + KY - 1;          // input rows of the footprint
  static constexpr int TXI = TX + KX - 1;          // input columns of the footprint
  static constexpr int XH = (W1 + 7) / 8 * 8;      // aligned left halo loaded
  static constexpr int BXW = ((XH + TX + W2) + 7) / 8 * 8;  // box width (elements)
  static constexpr int COFF = XH - W1;             // column 0 of the footprint in the box
  static constexpr int VSP = TXI + 4;              // padded row of the vertical-sum buffer
  static constexpr int LANES = TX / 4;             // lanes with output columns (4 each)
  static_assert(BXW <= 256, "box too wide");
  static_assert(TX % 8 == 0 && TX <= 128, "footprint width must be a multiple of 8 of at most 128");
};

constexpr int kTY3 = 8;  // output rows of a footprint
// Output columns of a footprint: as many as keep the TX + K - 1 input columns
// of the vertical pass within the CTA's 128 threads (one column each, no
// second round for a few threads), a multiple of 8 so that every footprint's
// TMA box starts on a 16-byte boundary for both element sizes.
template <int K>
constexpr int tx3() {
  return K3_THREADS - (K - 1 + 7) / 8 * 8;
}

// Item exactness: 0 if some in-volume value of cells [z0, z1] x [y0, y1] x
// [x0, x1] does not convert exactly under the item's maps (every thread of the
// CTA calls it; the answer is the CTA's).  Thread t reads column x0 + t of
// every row (coalesced), four rows' loads in flight at a time.
static __device__ __noinline__ int item_exact_3d(const float* gx, const float* gy, long long pz, long long py, int z0,
                                                 int z1, int y0, int y1, int x0, int x1, FxMap qx, FxMap qy) {
  bool ok = true;
  const int x = x0 + (int)threadIdx.x;
  if (x <= x1) {
    for (int z = z0; z <= z1; z++) {
      for (int y = y0; y <= y1; y += 4) {
        float a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const long long o = (long long)z * pz + (long long)min(y + u, y1) * py + x;
          a[u] = gx[o];
          b[u] = gy[o];
        }
#pragma unroll
        for (int u = 0; u < 4; u++) ok = ok && fx_on_grid(a[u], qx) && fx_on_grid(b[u], qy);
      }
    }
  }
  return __syncthreads_or(!ok) ? 0 : 1;
}

// Geometry a fix-up needs (passed by value).
struct Fix3D {
  const float* gx;
  const float* gy;
  long long pz, py;
  int Z, H, W, hz1, hz2, h1, h2, w1, w2, sz, sy, sx;
  float* out;
  long long opz, opy;
};

// Recompute the window of centre (zc, yc, xc) from its cells, the whole warp
// together (fx_box_warp), and store it over the earlier result.
static __device__ __noinline__ void fix_window_warp_3d(const Fix3D& f, int zc, int yc, int xc) {
  FxBox b;
  b.gx = f.gx;
  b.gy = f.gy;
  b.pz = f.pz;
  b.py = f.py;
  b.z0 = max(zc - f.hz1, 0);
  b.z1 = min(zc + f.hz2, f.Z - 1);
  b.y0 = max(yc - f.h1, 0);
  b.y1 = min(yc + f.h2, f.H - 1);
  b.x0 = max(xc - f.w1, 0);
  b.x1 = min(xc + f.w2, f.W - 1);
  const float c = fx_box_warp(b, nullptr);
  if ((threadIdx.x & 31) == 0) f.out[(long long)(zc / f.sz) * f.opz + (long long)(yc / f.sy) * f.opy + xc / f.sx] = c;
}

// The windows the wide re-march of an item could not certify (every thread
// of the CTA calls it): each listed window (n <= cap entries: centre plane
// << 10 | thread << 3 | bit 4a + c), or, if the list overflowed, every output
// window of the item (planes [zc0, zc1), rows [y0, y0 + ty), columns
// [x0, x0 + tx)), is recomputed by one warp from its own cells.
static __device__ __noinline__ void fix_listed_3d(Fix3D f, const uint64_t* list, int n, int cap, int y0, int x0,
                                                  int zc0, int zc1, int ty, int tx, uint32_t* status) {
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (n <= cap) {
    for (int i = warp; i < n; i += nw) {
      const uint64_t e = list[i];
      const int zc = (int)(e >> 10), t = (int)(e >> 3) & 127, bit = (int)(e & 7);
      fix_window_warp_3d(f, zc, y0 + (t >> 5) * 2 + (bit >> 2), x0 + 4 * (t & 31) + (bit & 3));
    }
    if (threadIdx.x == 0) atomicAdd(status + ST_FALLBACK, (uint32_t)n);
    return;
  }
  const long long total = (long long)(zc1 - zc0) * ty * tx;
  for (long long i = warp; i < total; i += nw) {
    const int xc = x0 + (int)(i % tx), yc = y0 + (int)((i / tx) % ty), zc = zc0 + (int)(i / ((long long)tx * ty));
    if (xc < f.W && yc < f.H && zc % f.sz == 0 && yc % f.sy == 0 && xc % f.sx == 0) fix_window_warp_3d(f, zc, yc, xc);
  }
}

#ifndef SWC_K3D_MINB
#define SWC_K3D_MINB 3  // resident CTAs per SM the 3-D kernel is compiled for
#endif
// WIDE = false: the kernel for every item (uint16, or float32 with the 22-bit
// item map).  WIDE = true (float32 only): the second tier, run on the items
// the first kernel listed, with a finer map of the item's range, fx_wide
// (up to 26 bits; rho = 1/2), 64-bit first-moment sums and Eq. 2 in 128-bit
// integers; windows that still fail are recomputed from their own cells.
template <int TY, int TX, int KY, int KX, bool WIDE>
__global__ void __launch_bounds__(K3_THREADS, SWC_K3D_MINB) k3d_kernel(const __grid_constant__ K3DParams p) {
  using G = Geo3D<TY, TX, KY, KX>;
  using T1 = std::conditional_t<WIDE, uint64_t, uint32_t>;  // first-moment sums
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int esz = p.is_f32 ? 4 : 2;
  const size_t plane_bytes = (size_t)G::TYI * G::BXW * esz;   // one channel of one plane
  const size_t plane_stride = (plane_bytes + 127) / 128 * 128;  // TMA destinations are 128-byte aligned
  const size_t slot_bytes = 2 * plane_stride;                   // x, then y
  const int yoff = (int)(plane_stride / esz);                    // y channel, in elements
  // slots: 0 entering plane, 1 leaving plane (the range pass of float32
  // items alternates between both)
  unsigned char* slots = smem_raw;
  uint32_t* VS = reinterpret_cast<uint32_t*>(smem_raw + 2 * slot_bytes);  // [8][TY][VSP]
  uint64_t* bar = reinterpret_cast<uint64_t*>(VS + 8 * TY * G::VSP);      // 2 mbarriers (4 reserved)
  static_assert(G::TXI <= K3_THREADS, "one input column per thread");
  __shared__ float red[4][K3_THREADS / 32];
  // item constants, uniform over the CTA, kept here rather than in registers:
  // the float32 maps, the value G of an off-volume cell, the certificate's
  // rounding bounds (0 once the item converts exactly; uint16 is exact)
  __shared__ FxMap sh_qx, sh_qy;
  __shared__ FxWide sh_wx, sh_wy;
  __shared__ float sh_rho[2];
  // windows whose certificate failed during the item's z-march
  constexpr int kPendCap = 384;
  __shared__ uint64_t sh_pend[kPendCap];
  __shared__ int sh_npend;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (tid == 0) {
    for (int b = 0; b < 4; b++) mbar_init(bar + b, 1);
    fence_mbar_init();
    if (p.use_tma) {
      prefetch_tmap(&p.tmx);
      prefetch_tmap(&p.tmy);
    }
  }
  __syncthreads();
  uint32_t phase_bits = 0;  // parity of each of the 4 barriers

  const int n_iter = WIDE ? *p.redo_count : p.n_items;
  for (int it = blockIdx.x; it < n_iter; it += gridDim.x) {
    const int item = WIDE ? p.redo_items[it] : it;
    int rem = item;
    const int xb = rem % p.nxb; rem /= p.nxb;
    const int yb = rem % p.nyb; rem /= p.nyb;
    const int zbk = rem;
    const int x0 = xb * TX, y0 = yb * TY;              // first centre column / row of the footprint
    const int zc0 = zbk * p.TZ;                        // first centre plane
    const int zc1 = min(zc0 + p.TZ, p.Z);
    const int ze0 = zc0 - p.hz1;                       // first entering plane
    const int nsteps = (zc1 - zc0) + p.kz - 1;
    const int bx = x0 - G::XH, by = y0 - G::H1;        // box origin

    auto issue = [&](int slot, int z) {  // thread 0 only
      uint64_t* b = bar + slot;
      unsigned char* d = slots + slot * slot_bytes;
      mbar_arrive_expect_tx(b, (uint32_t)(2 * plane_bytes));
      tma_load_3d(d, &p.tmx, bx, by, z, b);
      tma_load_3d(d + plane_stride, &p.tmy, bx, by, z, b);
    };
    auto wait_slot = [&](int slot) -> bool {
      if (!p.use_tma) return true;
      const bool ok = mbar_wait_bounded(bar + slot, (phase_bits >> slot) & 1u, p.status);
      phase_bits ^= (1u << slot);
      return ok;
    };
    // plain-load variant of issue(): the whole CTA copies the box (zero fill
    // off the volume); the caller synchronises before use
    auto load_plain = [&](int slot, int z) {
      unsigned char* d = slots + slot * slot_bytes;
      const bool z_ok = z >= 0 && z < p.Z;
      for (int e = tid; e < G::TYI * G::BXW; e += K3_THREADS) {
        const int r = e / G::BXW, cidx = e - r * G::BXW;
        const int gy = by + r, gxx = bx + cidx;
        const bool ok = z_ok && gy >= 0 && gy < p.H && gxx >= 0 && gxx < p.W;
        const long long g = (long long)z * p.ipz + (long long)gy * p.ipy + gxx;
        if (esz == 4) {
          reinterpret_cast<float*>(d)[e] = ok ? __ldg((const float*)p.gx + g) : 0.0f;
          reinterpret_cast<float*>(d + plane_stride)[e] = ok ? __ldg((const float*)p.gy + g) : 0.0f;
        } else {
          reinterpret_cast<uint16_t*>(d)[e] = ok ? __ldg((const uint16_t*)p.gx + g) : (uint16_t)0;
          reinterpret_cast<uint16_t*>(d + plane_stride)[e] = ok ? __ldg((const uint16_t*)p.gy + g) : (uint16_t)0;
        }
      }
    };

    if (tid == 0) sh_npend = 0;  // (ordered by the barriers of the range pass or the first step)
    // ---- float32: one fixed-point map for the item (pass over its planes)
    if (p.is_f32) {
      float xlo = 3.0e38f, xhi = -3.0e38f, ylo = 3.0e38f, yhi = -3.0e38f;
      if (tid == 0 && p.use_tma) {
        fence_proxy_async_smem();
        issue(0, ze0);
      }
      for (int s = 0; s < nsteps; s++) {
        if (!p.use_tma) {
          load_plain(s & 1, ze0 + s);
          __syncthreads();
        } else if (tid == 0 && s + 1 < nsteps) {
          fence_proxy_async_smem();
          issue((s + 1) & 1, ze0 + s + 1);
        }
        if (!wait_slot(s & 1)) return;
        const int z = ze0 + s;
        // thread tid scans input column tid of the footprint down its rows
        const int gxx = x0 - G::W1 + tid;
        if (z >= 0 && z < p.Z && tid < G::TXI && gxx >= 0 && gxx < p.W) {
          const float* px = reinterpret_cast<const float*>(slots + (s & 1) * slot_bytes) + G::COFF + tid;
          const float* py = px + yoff;
#pragma unroll
          for (int r = 0; r < G::TYI; r++) {
            const int gy = by + r;
            if (gy >= 0 && gy < p.H) {
              const float a = px[r * G::BXW], b = py[r * G::BXW];
              xlo = fminf(xlo, a); xhi = fmaxf(xhi, a); ylo = fminf(ylo, b); yhi = fmaxf(yhi, b);
            }
          }
        }
        __syncthreads();
      }
      // block reduction
      for (int o = 16; o > 0; o >>= 1) {
        xlo = fminf(xlo, __shfl_xor_sync(0xffffffffu, xlo, o));
        xhi = fmaxf(xhi, __shfl_xor_sync(0xffffffffu, xhi, o));
        ylo = fminf(ylo, __shfl_xor_sync(0xffffffffu, ylo, o));
        yhi = fmaxf(yhi, __shfl_xor_sync(0xffffffffu, yhi, o));
      }
      if (lane == 0) {
        red[0][warp] = xlo; red[1][warp] = xhi; red[2][warp] = ylo; red[3][warp] = yhi;
      }
      __syncthreads();
      xlo = red[0][0]; xhi = red[1][0]; ylo = red[2][0]; yhi = red[3][0];
      for (int w = 1; w < K3_THREADS / 32; w++) {
        xlo = fminf(xlo, red[0][w]); xhi = fmaxf(xhi, red[1][w]);
        ylo = fminf(ylo, red[2][w]); yhi = fmaxf(yhi, red[3][w]);
      }
      __syncthreads();
      if (tid == 0) {
        if constexpr (WIDE) {
          const long long nfull = (long long)p.kz * KY * KX;
          sh_wx = fx_wide(xlo, xhi, nfull);
          sh_wy = fx_wide(ylo, yhi, nfull);
          sh_rho[0] = sh_rho[1] = 0.5f;
        } else {
          const FxMap qx = fx_make(xlo, xhi, p.qbits), qy = fx_make(ylo, yhi, p.qbits);
          sh_qx = qx;
          sh_qy = qy;
          sh_rho[0] = qx.rho;
          sh_rho[1] = qy.rho;
        }
      }
    } else if (tid == 0) {
      sh_rho[0] = sh_rho[1] = 0.0f;
    }
    // (the first step's barrier after the vertical pass orders these stores
    // before their first reads in step 4)

    // ---- the z-march
    T1 V0[2][4], V1[2][4];
    uint64_t V2[2][4], V3[2][4], V4[2][4];
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
      for (int c = 0; c < 4; c++) {
        V0[a][c] = V1[a][c] = 0u;
        V2[a][c] = V3[a][c] = V4[a][c] = 0ull;
      }
    // entering plane of step s in slot 0, leaving plane (step s >= kz) in
    // slot 1; the copies of step s + 1 are issued as soon as the vertical
    // pass of step s has read both, so they overlap the horizontal pass
    if (tid == 0 && p.use_tma) {
      fence_proxy_async_smem();
      issue(0, ze0);  // kz >= 1: no leaving plane at step 0
    }
    for (int s = 0; s < nsteps; s++) {
      const int ze = ze0 + s, zl = ze - p.kz;
      const bool has_leave = s >= p.kz;
      if (!p.use_tma) {
        load_plain(0, ze);
        if (has_leave) load_plain(1, zl);
        __syncthreads();
      }
      if (!wait_slot(0)) return;
      if (has_leave && !wait_slot(1)) return;
      const bool ze_ok = ze >= 0 && ze < p.Z;
      const bool zl_ok = has_leave && zl >= 0 && zl < p.Z;
      const unsigned char* se = slots;
      const unsigned char* sl = slots + slot_bytes;

      // vertical pass: thread per input column; a footprint whose input rows
      // all lie in the volume takes a variant without the per-row test
      auto vcol = [&](int c, auto y_in_tag) {
        constexpr bool Y_IN = decltype(y_in_tag)::value;
        const int gxx = x0 - G::W1 + c;
        const bool col_ok = gxx >= 0 && gxx < p.W;
        const bool ue = col_ok && ze_ok, ul = col_ok && zl_ok;
        // float32: a zero scale and the plain rounding constant convert
        // off-volume cells to X = 0
        const float mx = sh_qx.msub, my = sh_qy.msub;
        const float fse_x = ue ? sh_qx.s : 0.f, fsl_x = ul ? sh_qx.s : 0.f;
        const float fse_y = ue ? sh_qy.s : 0.f, fsl_y = ul ? sh_qy.s : 0.f;
        const float fce_x = ue ? sh_qx.C : kFxMagic, fcl_x = ul ? sh_qx.C : kFxMagic;
        const float fce_y = ue ? sh_qy.C : kFxMagic, fcl_y = ul ? sh_qy.C : kFxMagic;
        uint32_t P0 = 0u, P1 = 0u;
        uint64_t P2 = 0ull, P3 = 0ull, P4 = 0ull;
        uint32_t S0[TY], S1[TY];
        uint64_t S2[TY], S3[TY], S4[TY];
#pragma unroll
        for (int r = 0; r < G::TYI; r++) {
          const int gy = by + r;
          const bool row_ok = Y_IN || (gy >= 0 && gy < p.H);
          const int idx = r * G::BXW + G::COFF + c;
          int Xe, Xl, Ye, Yl;
          if constexpr (WIDE) {
            // X = round(x s) - M in 32 bits (fx_wide); off-volume cells are
            // absent (X = 0)
            const float* pe = reinterpret_cast<const float*>(se);
            const float* pl = reinterpret_cast<const float*>(sl);
            const bool ie = ue && row_ok, il = ul && row_ok;
            Xe = ie ? __float2int_rn((pe[idx] - sh_wx.sub) * sh_wx.s) - sh_wx.moff : 0;
            Ye = ie ? __float2int_rn((pe[yoff + idx] - sh_wy.sub) * sh_wy.s) - sh_wy.moff : 0;
            Xl = il ? __float2int_rn((pl[idx] - sh_wx.sub) * sh_wx.s) - sh_wx.moff : 0;
            Yl = il ? __float2int_rn((pl[yoff + idx] - sh_wy.sub) * sh_wy.s) - sh_wy.moff : 0;
          } else if (p.is_f32) {
            const float* pe = reinterpret_cast<const float*>(se);
            const float* pl = reinterpret_cast<const float*>(sl);
            const float xl = has_leave ? pl[idx] : 0.f, yl = has_leave ? pl[yoff + idx] : 0.f;
            auto cv = [&](float v, float m, float sc, float cc) {
              return __float_as_int(fmaf(v - m, row_ok ? sc : 0.f, row_ok ? cc : kFxMagic)) - 0x4B400000;
            };
            Xe = cv(pe[idx], mx, fse_x, fce_x);
            Ye = cv(pe[yoff + idx], my, fse_y, fce_y);
            Xl = cv(xl, mx, fsl_x, fcl_x);
            Yl = cv(yl, my, fsl_y, fcl_y);
          } else {
            const uint16_t* pe = reinterpret_cast<const uint16_t*>(se);
            const uint16_t* pl = reinterpret_cast<const uint16_t*>(sl);
            Xe = (ue && row_ok) ? (int)pe[idx] : 0;
            Ye = (ue && row_ok) ? (int)pe[yoff + idx] : 0;
            Xl = (ul && row_ok) ? (int)pl[idx] : 0;
            Yl = (ul && row_ok) ? (int)pl[yoff + idx] : 0;
          }
          const int D = (int)((uint32_t)Xe - (uint32_t)Xl), S = (int)((uint32_t)Xe + (uint32_t)Xl);
          const int Dy = (int)((uint32_t)Ye - (uint32_t)Yl), Sy = (int)((uint32_t)Ye + (uint32_t)Yl);
          P0 += (uint32_t)D;
          P1 += (uint32_t)Dy;
          P2 += (uint64_t)((long long)D * S);
          P3 += (uint64_t)((long long)Dy * Sy);
          P4 += (uint64_t)((long long)D * Ye) + (uint64_t)((long long)Xl * Dy);
          if (r <= TY - 2) {
            S0[r + 1] = P0; S1[r + 1] = P1; S2[r + 1] = P2; S3[r + 1] = P3; S4[r + 1] = P4;
          }
          if (r >= KY - 1) {
            const int y = r - (KY - 1);
            const uint32_t v0 = P0 - (y >= 1 ? S0[y] : 0u), v1 = P1 - (y >= 1 ? S1[y] : 0u);
            const uint64_t v2 = P2 - (y >= 1 ? S2[y] : 0ull), v3 = P3 - (y >= 1 ? S3[y] : 0ull);
            const uint64_t v4 = P4 - (y >= 1 ? S4[y] : 0ull);
            const int base = y * G::VSP + c;
            const int plane = TY * G::VSP;
            VS[0 * plane + base] = v0;
            VS[1 * plane + base] = v1;
            VS[2 * plane + base] = (uint32_t)v2;
            VS[3 * plane + base] = (uint32_t)(v2 >> 32);
            VS[4 * plane + base] = (uint32_t)v3;
            VS[5 * plane + base] = (uint32_t)(v3 >> 32);
            VS[6 * plane + base] = (uint32_t)v4;
            VS[7 * plane + base] = (uint32_t)(v4 >> 32);
          }
        }
      };
      const bool y_in = by >= 0 && by + G::TYI <= p.H;
      for (int c = tid; c < G::TXI; c += K3_THREADS) {
        if (y_in)
          vcol(c, std::true_type{});
        else
          vcol(c, std::false_type{});
      }
      __syncthreads();
      // both slots are free: request step s + 1
      if (tid == 0 && p.use_tma && s + 1 < nsteps) {
        fence_proxy_async_smem();
        issue(0, ze + 1);
        if (s + 1 >= p.kz) issue(1, ze + 1 - p.kz);
      }

      // horizontal pass: warp -> 2 output rows, lane -> 4 output columns
      // (lanes past the footprint's TX columns have none).  Strided plans
      // (a variant of their own, so that unit strides pay nothing) skip rows
      // that are not output rows and update the running sums of output
      // columns only (col_mask bit c: column xc0 + c is one).
      const bool lane_on = lane < G::LANES;
      auto hpass = [&](auto strided_tag) {
        constexpr bool STRIDED = decltype(strided_tag)::value;
        uint32_t col_mask = 0xFu;
        if constexpr (STRIDED) {
          col_mask = 0u;
#pragma unroll
          for (int c = 0; c < 4; c++) col_mask |= ((x0 + 4 * lane + c) % p.sx == 0) ? (1u << c) : 0u;
        }
#pragma unroll
        for (int a = 0; a < 2; a++) {
          if (!lane_on) break;
          const int y = warp * 2 + a;
          if (STRIDED && (y0 + y) % p.sy != 0) continue;
          T1 Q0 = 0u, Q1 = 0u;
          uint64_t Q2 = 0ull, Q3 = 0ull, Q4 = 0ull;
          T1 R0[4], R1[4];
          uint64_t R2[4], R3[4], R4[4];
          const int plane = TY * G::VSP;
#pragma unroll
          for (int e = 0; e < 4 + KX - 1; e++) {
            const int cidx = y * G::VSP + 4 * lane + e;
            // (wide: the ky-row sums of X fit int32; their kx-column sums may not)
            Q0 += WIDE ? (T1)(long long)(int)VS[0 * plane + cidx] : (T1)VS[0 * plane + cidx];
            Q1 += WIDE ? (T1)(long long)(int)VS[1 * plane + cidx] : (T1)VS[1 * plane + cidx];
            Q2 += (uint64_t)VS[2 * plane + cidx] | ((uint64_t)VS[3 * plane + cidx] << 32);
            Q3 += (uint64_t)VS[4 * plane + cidx] | ((uint64_t)VS[5 * plane + cidx] << 32);
            Q4 += (uint64_t)VS[6 * plane + cidx] | ((uint64_t)VS[7 * plane + cidx] << 32);
            if (e <= 2) {
              R0[e + 1] = Q0; R1[e + 1] = Q1; R2[e + 1] = Q2; R3[e + 1] = Q3; R4[e + 1] = Q4;
            }
            if (e >= KX - 1 && (!STRIDED || ((col_mask >> (e - (KX - 1))) & 1u))) {
              const int c = e - (KX - 1);
              V0[a][c] += Q0 - (c >= 1 ? R0[c] : (T1)0u);
              V1[a][c] += Q1 - (c >= 1 ? R1[c] : (T1)0u);
              V2[a][c] += Q2 - (c >= 1 ? R2[c] : 0ull);
              V3[a][c] += Q3 - (c >= 1 ? R3[c] : 0ull);
              V4[a][c] += Q4 - (c >= 1 ? R4[c] : 0ull);
            }
          }
        }
      };
      if (p.unit_stride)
        hpass(std::false_type{});
      else
        hpass(std::true_type{});

      // step 4 for the output plane whose window is complete: Eq. 2 from the
      // exact sums of window (a, c) with n in-volume cells; `fail` reports a
      // float32 window whose certificate does not hold
      const float rhox = sh_rho[0], rhoy = sh_rho[1];
      // quick certificate thresholds (rho n / 4.5e-6)^2 for the full window
      const float k0 = 4.9432e10f * (float)(p.kz * KY * KX) * (float)(p.kz * KY * KX);
      const float Kx = k0 * rhox * rhox, Ky = k0 * rhoy * rhoy;
      const bool f32 = p.is_f32 != 0;
      auto eval = [&](int a, int c, int cz, uint32_t n32, bool& fail) -> float {
        if constexpr (WIDE) {
          // sums of X^2 below 2^62 (fx_wide), first moments 64-bit: Eq. 2 in
          // 128-bit integers
          const __int128 n = n32;
          const long long s0 = (long long)V0[a][c], s1 = (long long)V1[a][c];
          const __int128 vx = n * (long long)V2[a][c] - (__int128)s0 * s0;
          const __int128 vy = n * (long long)V3[a][c] - (__int128)s1 * s1;
          const __int128 num = n * (long long)V4[a][c] - (__int128)s0 * s1;
          fail = !fx_certified(i128_to_f32(vx), i128_to_f32(vy), (float)n32, 0.5f, 0.5f);
          return fx_pearson128(num, vx, vy);
        }
        // exact in 64-bit modular arithmetic; the results are below 2^63
        const uint64_t n = n32;
        const uint64_t nq2 = n * V2[a][c], nq3 = n * V3[a][c];
        const uint64_t s0 = (uint64_t)(long long)(int)V0[a][c], s1 = (uint64_t)(long long)(int)V1[a][c];
        const long long vx = (long long)(nq2 - s0 * s0);
        const long long vy = (long long)(nq3 - s1 * s1);
        const long long num = (long long)(n * V4[a][c] - s0 * s1);
        const float fvx = i64_to_f32(vx), fvy = i64_to_f32(vy);
        // float32 certificate: the quick per-channel test, the precise sum
        // when it fails; the first moments read as int32 are exact while
        // n Sxx < 2^62 (a window beyond that fails)
        fail = false;
        if (f32) {
          const bool wide = ((nq2 | nq3) >> 62) != 0ull;
          fail = wide || !(fvx >= Kx && fvy >= Ky);
          if (fail && !wide) fail = !((float)n32 * (rhox * rsqrtf(fvx) + rhoy * rsqrtf(fvy)) <= 8.99e-6f);
        }
        // a zero variance makes num exactly 0, so 0 * rsqrt(0) = NaN
        return clamp1_nan(i64_to_f32(num) * rsqrtf(fvx * fvy));
      };
      // debug output of uint16 plans: the exact window sums of output (jz, jy, jx)
      auto emit = [&](int a, int c, int jz, int jy, int jx) {
        if (!WIDE && p.sums != nullptr) {
          long long* s5 = p.sums + 5 * (((long long)jz * p.OY + jy) * p.OX + jx);
          s5[0] = (int)V0[a][c];  // below 2^31 for uint16 windows of at most 32768 cells
          s5[1] = (int)V1[a][c];
          s5[2] = (long long)V2[a][c];
          s5[3] = (long long)V3[a][c];
          s5[4] = (long long)V4[a][c];
        }
      };
      uint32_t pending = 0;  // bit 4a + c: window whose certificate failed
      int zc_out = 0;
      if (!lane_on) {
      } else if (s >= p.kz - 1 && p.unit_stride) {
        // unit strides: output (z, y, x) = centre (z, y, x); 4 columns per lane
        const int zc = zc0 + (s - (p.kz - 1));
        zc_out = zc;
        const int cz = min(zc + p.hz2, p.Z - 1) - max(zc - p.hz1, 0) + 1;
#pragma unroll
        for (int a = 0; a < 2; a++) {
          const int yc = y0 + warp * 2 + a;
          if (yc >= p.H) continue;
          const int cy = min(yc + G::H2, p.H - 1) - max(yc - G::H1, 0) + 1;
          float* orow = p.out + (long long)zc * p.opz + (long long)yc * p.opy;
          const int xc0 = x0 + 4 * lane;
          float res[4];
#pragma unroll
          for (int c = 0; c < 4; c++) {
            const int xc = xc0 + c;
            const int cx = max(min(xc + G::W2, p.W - 1) - max(xc - G::W1, 0) + 1, 0);
            bool f;
            res[c] = eval(a, c, cz, (uint32_t)(cz * cy * cx), f);
            if (f && xc < p.W) pending |= 1u << (4 * a + c);
            if (!f32 && xc < p.W) emit(a, c, zc, yc, xc);
          }
          if (p.vec_store && xc0 + 3 < p.W) {
            stg128(orow + xc0, res[0], res[1], res[2], res[3]);
          } else {
#pragma unroll
            for (int c = 0; c < 4; c++)
              if (xc0 + c < p.W) orow[xc0 + c] = res[c];
          }
        }
      } else if (s >= p.kz - 1) {
        const int zc = zc0 + (s - (p.kz - 1));
        zc_out = zc;
        if (zc % p.sz == 0) {
          const int cz = min(zc + p.hz2, p.Z - 1) - max(zc - p.hz1, 0) + 1;
#pragma unroll
          for (int a = 0; a < 2; a++) {
            const int yc = y0 + warp * 2 + a;
            if (yc >= p.H || yc % p.sy != 0) continue;
            const int cy = min(yc + G::H2, p.H - 1) - max(yc - G::H1, 0) + 1;
            float* orow = p.out + (long long)(zc / p.sz) * p.opz + (long long)(yc / p.sy) * p.opy;
#pragma unroll
            for (int c = 0; c < 4; c++) {
              const int xc = x0 + 4 * lane + c;
              if (xc >= p.W || xc % p.sx != 0) continue;
              const int cx = min(xc + G::W2, p.W - 1) - max(xc - G::W1, 0) + 1;
              bool f;
              orow[xc / p.sx] = eval(a, c, cz, (uint32_t)(cz * cy * cx), f);
              if (f) pending |= 1u << (4 * a + c);
              if (!f32) emit(a, c, zc / p.sz, yc / p.sy, xc / p.sx);
            }
          }
        }
      }
      // VS and the ring slots are reused next step (this is the step's barrier)
      for (; pending; pending &= pending - 1) {  // rare: list the failing windows
        const int k = atomicAdd(&sh_npend, 1);
        if (k < kPendCap) sh_pend[k] = ((uint64_t)zc_out << 10) | ((uint64_t)tid << 3) | (uint64_t)(__ffs(pending) - 1);
      }
      __syncthreads();  // VS and the ring slots are reused next step
    }
    // the item's failing windows (float32 only), once its z-march is done
    if constexpr (WIDE) {
      // every window of the item was rewritten; the listed ones are recomputed
      if (tid == 0) {
        auto multiples = [](int a, int b, int st) { return (b + st - 1) / st - (a + st - 1) / st; };  // in [a, b)
        const long long outs = (long long)multiples(zc0, zc1, p.sz) * multiples(y0, min(y0 + TY, p.H), p.sy) *
                               multiples(x0, min(x0 + TX, p.W), p.sx);
        atomicAdd(p.status + ST_FALLBACK, (uint32_t)outs);
      }
      if (sh_npend > 0) {
        const Fix3D fx{(const float*)p.gx, (const float*)p.gy, p.ipz, p.ipy, p.Z, p.H, p.W, p.hz1, p.hz2,
                       G::H1, G::H2, G::W1, G::W2, p.sz, p.sy, p.sx, p.out, p.opz, p.opy};
        fix_listed_3d(fx, sh_pend, sh_npend, kPendCap, y0, x0, zc0, zc1, TY, TX, p.status);
      }
      __syncthreads();  // the list and the item constants are reset by the next item
    } else if (p.is_f32 && sh_npend > 0) {
      // unless the item's values convert exactly (then every result stands),
      // list the item for the wide kernel
      if (!item_exact_3d((const float*)p.gx, (const float*)p.gy, p.ipz, p.ipy, max(ze0, 0),
                         min(ze0 + nsteps, p.Z) - 1, max(by, 0), min(by + G::TYI, p.H) - 1, max(x0 - G::W1, 0),
                         min(x0 - G::W1 + G::TXI, p.W) - 1, sh_qx, sh_qy) &&
          tid == 0)
        p.redo_items[atomicAdd(p.redo_count, 1)] = item;
      __syncthreads();  // the list and the item constants are reset by the next item
    }
  }
}

}  // namespace swc
