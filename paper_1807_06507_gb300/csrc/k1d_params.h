// k1d_params.h -- parameters of the fused 1-D kernel (host and device).
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace swc {

struct K1DParams {
  CUtensorMap tmx;  // 1-D maps: dims {N}, box {256}
  CUtensorMap tmy;
  long long N;       // series length
  int k, h1, h2;     // window and its extents before/after the centre
  int stride;
  long long n_out;   // ceil(N / stride)
  long long n_items; // chunks of (warps per CTA) * 32 * M1 outputs
  int span;          // cells loaded per chunk (= nbox * 256)
  int nbox;          // TMA boxes per channel per chunk
  int q, r;          // k = q * (M1 * stride) + r
  int nseg;          // segments of M1*stride cells a warp sums (<= 64)
  int is_f32;
  int qbits;         // float32 fixed-point magnitude bits
  const void* gx;    // plain-load fallback (unaligned bases); NULL when TMA loads
  const void* gy;
  const void* rx;    // the series themselves (always set: float32 windows that
  const void* ry;    //   fail their certificate are recomputed from them)
  float* out;
  long long* sums;   // optional (uint16): 5 int64 per output, Sx Sy Sxx Syy Sxy
  uint32_t* status;
  // float32: chunks whose windows the chunk's map left uncertified (the
  // first launch appends them; the wide launch re-slides them)
  int* redo_count;
  long long* redo_items;
};

}  // namespace swc
