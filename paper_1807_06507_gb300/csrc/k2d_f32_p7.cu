// k2d_f32_p7.cu -- fused 2-D float32 kernel instances for window widths 29 and 31
// (each with and without TMA, for the three second-tier placements).
#include "k2d_f32_kern.cuh"

namespace swc {

SWC_K2DF_PART(k2d_f32_launch_p7, 29, 31)

}  // namespace swc
