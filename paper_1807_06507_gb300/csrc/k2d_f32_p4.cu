// k2d_f32_p4.cu -- fused 2-D float32 kernel instances for window widths 17 and 19
// (each with and without TMA, for the three second-tier placements).
#include "k2d_f32_kern.cuh"

namespace swc {

SWC_K2DF_PART(k2d_f32_launch_p4, 17, 19)

}  // namespace swc
