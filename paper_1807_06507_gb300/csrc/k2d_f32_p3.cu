// k2d_f32_p3.cu -- fused 2-D float32 kernel instances for window widths 25, 27, 29, 31.
#include "k2d_f32_kern.cuh"

namespace swc {

SWC_K2DF_PART(k2d_f32_launch_p3, 25, 27, 29, 31)

}  // namespace swc
