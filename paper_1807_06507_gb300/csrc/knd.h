// knd.h -- parameters of the general n-dimensional path (host and device).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace swc {

constexpr int KND_MAXDIM = 8;

struct KNDParams {
  int ndim;
  long long shape[KND_MAXDIM];   // cells per dimension (C order)
  long long inner[KND_MAXDIM];   // cells between neighbours along d in the work buffers
  long long ipitch[KND_MAXDIM];  // input element pitches
  int h1[KND_MAXDIM], h2[KND_MAXDIM];  // window extents before / after the centre
  int stride[KND_MAXDIM];
  long long oshape[KND_MAXDIM];  // ceil(shape / stride)
  long long ncell, nout;
  int nstreams;                  // 5, or 6 with the missing-cell count (1 when mask_only)
  int is_f32, paper, sat, qbits;
  int mask_only;                 // the paper's convention after a fused kernel: only the
                                 //   missing-cell count is summed; the finalize writes -2 where
                                 //   the window passes an edge or holds a missing cell and leaves
                                 //   every other output as the fused kernel wrote it
  const void* x;
  const void* y;
  float* out;                    // contiguous output
  long long* sums;               // optional: 5 int64 per output (uint16)
  long long* buf[2];             // nstreams x ncell int64 each (ping-pong)
  long long* segs;               // cumulative-sum ablation: segment totals, nstreams x (ncell / 128 + ncell / N_d)
  float* scratch;                // range of x and y, exactness flag (8 words)
  uint32_t* status;
};

// Queue the whole path (range, conversion, one pass per dimension, finalize).
cudaError_t knd_launch(const KNDParams& p, int sms, cudaStream_t st);

}  // namespace swc
