// k2d_f32.cu -- geometry and launch dispatch of the fused 2-D float32
// correlation (one warp per CTA, persistent over work items); the kernel's
// instances live in k2d_f32_p0.cu .. k2d_f32_p7.cu.
#include "k2d_f32.cuh"
#include "launch.h"

namespace swc {

template <int M, int KW>
static void geo(Geo2DInfo* g) {
  using G = Geo2DF<M, KW>;
  g->M = M;
  g->KW = KW;
  g->HALO = G::HALO;
  g->RW = G::RW;
  g->RWS = G::RWS;
  g->TAIL = G::TAIL;
}

#define SWC_K2DF_CASES(X) X(8, 1) X(8, 3) X(8, 5) X(8, 7) X(8, 9) X(8, 11) X(8, 13) X(8, 15) X(8, 17) \
  X(8, 19) X(8, 21) X(8, 23) X(8, 25) X(8, 27) X(8, 29) X(8, 31)

bool k2d_f32_geometry(int kw, Geo2DInfo* g) {
  switch (kw) {
#define X(M, KW) \
  case KW:       \
    geo<M, KW>(g); \
    return true;
    SWC_K2DF_CASES(X)
#undef X
    default:
      return false;
  }
}

cudaError_t k2d_f32_launch(int kw, const K2DParams& p, int grid, size_t smem, cudaStream_t st, bool tma, int tier) {
  if (kw < 1 || kw > 31 || kw % 2 == 0) return cudaErrorInvalidValue;
  switch ((kw - 1) / 4) {  // the part holding this width
    case 0: return k2d_f32_launch_p0(kw, p, grid, smem, st, tma, tier);
    case 1: return k2d_f32_launch_p1(kw, p, grid, smem, st, tma, tier);
    case 2: return k2d_f32_launch_p2(kw, p, grid, smem, st, tma, tier);
    case 3: return k2d_f32_launch_p3(kw, p, grid, smem, st, tma, tier);
    case 4: return k2d_f32_launch_p4(kw, p, grid, smem, st, tma, tier);
    case 5: return k2d_f32_launch_p5(kw, p, grid, smem, st, tma, tier);
    case 6: return k2d_f32_launch_p6(kw, p, grid, smem, st, tma, tier);
    default: return k2d_f32_launch_p7(kw, p, grid, smem, st, tma, tier);
  }
}

}  // namespace swc
