// kbatched_f32_p0.cu -- batched float32 kernel instances for window widths 1 to 15.
#include "kbatched_f32_kern.cuh"

namespace swc {

SWC_KB32_PART(p0, 1, 3, 5, 7, 9, 11, 13, 15)

}  // namespace swc
