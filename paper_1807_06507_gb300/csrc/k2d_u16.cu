// k2d_u16.cu -- kernel entry points and instantiations of the fused 2-D
// uint16 correlation (one warp per CTA, persistent over work items).
#include "k2d_u16.cuh"
#include "devonce.h"
#include "launch.h"

namespace swc {

#ifndef SWC_K2D_WIDE
#define SWC_K2D_WIDE false
#endif

template <int M, int KW, bool TMA>
static cudaError_t launch_tma(const K2DParams& p, int grid, size_t smem, cudaStream_t st) {
  static std::atomic<uint64_t> attr_done{0};  // one bit per device
  cudaError_t e = once_per_device(attr_done, [] {
    return cudaFuncSetAttribute(k2d_u16_kernel<M, KW, TMA, SWC_K2D_WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  if (e != cudaSuccess) return e;
  k2d_u16_kernel<M, KW, TMA, SWC_K2D_WIDE><<<grid, 32, smem, st>>>(p);
  return cudaGetLastError();
}

template <int M, int KW>
static cudaError_t launch_one(const K2DParams& p, int grid, size_t smem, cudaStream_t st, bool tma) {
  return tma ? launch_tma<M, KW, true>(p, grid, smem, st) : launch_tma<M, KW, false>(p, grid, smem, st);
}

template <int M, int KW>
static void geo(Geo2DInfo* g) {
  using G = Geo2D<M, KW>;
  g->M = M;
  g->KW = KW;
  g->HALO = G::HALO;
  g->RW = G::RW;
  g->RWS = G::RWS;
  g->TAIL = G::TAIL;
}

#define SWC_K2D_CASES(X) X(8, 1) X(8, 3) X(8, 5) X(8, 7) X(8, 9) X(8, 11) X(8, 13) X(8, 15) X(8, 17) \
  X(8, 19) X(8, 21) X(8, 23) X(8, 25) X(8, 27) X(8, 29) X(8, 31)

bool k2d_u16_geometry(int kw, Geo2DInfo* g) {
  switch (kw) {
#define X(M, KW) \
  case KW:       \
    geo<M, KW>(g); \
    return true;
    SWC_K2D_CASES(X)
#undef X
    default:
      return false;
  }
}

cudaError_t k2d_u16_launch_wide(int kw, const K2DParams& p, int grid, size_t smem, cudaStream_t st, bool tma);
int k2d_u16_blocks_wide(int kw, size_t smem);

int k2d_u16_blocks_per_sm(int kw, bool wide, size_t smem) {
  if (wide) return k2d_u16_blocks_wide(kw, smem);
  int b = 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (kw) {
#define X(M, KW)                                                                                      \
  case KW:                                                                                            \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k2d_u16_kernel<M, KW, true, false>, 32, smem); \
    break;
    SWC_K2D_CASES(X)
#undef X
    default:
      break;
  }
  return e == cudaSuccess ? b : 0;
}

static cudaError_t k2d_u16_launch_narrow(int kw, const K2DParams& p, int grid, size_t smem, cudaStream_t st,
                                         bool tma) {
  switch (kw) {
#define X(M, KW) \
  case KW:       \
    return launch_one<M, KW>(p, grid, smem, st, tma);
    SWC_K2D_CASES(X)
#undef X
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t k2d_u16_launch(int kw, const K2DParams& p, int grid, size_t smem, cudaStream_t st, bool tma) {
  return p.sc.wide ? k2d_u16_launch_wide(kw, p, grid, smem, st, tma) : k2d_u16_launch_narrow(kw, p, grid, smem, st, tma);
}

}  // namespace swc
