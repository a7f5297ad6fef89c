// k2d_f32_p2.cu -- fused 2-D float32 kernel instances for window widths 17, 19, 21, 23.
#include "k2d_f32_kern.cuh"

namespace swc {

SWC_K2DF_PART(k2d_f32_launch_p2, 17, 19, 21, 23)

}  // namespace swc
