// k2d_f32_p1.cu -- fused 2-D float32 kernel instances for window widths 9, 11, 13, 15.
#include "k2d_f32_kern.cuh"

namespace swc {

SWC_K2DF_PART(k2d_f32_launch_p1, 9, 11, 13, 15)

}  // namespace swc
