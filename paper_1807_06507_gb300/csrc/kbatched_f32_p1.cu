// kbatched_f32_p1.cu -- batched float32 kernel instances for window widths 17 to 31.
#include "kbatched_f32_kern.cuh"

namespace swc {

SWC_KB32_PART(p1, 17, 19, 21, 23, 25, 27, 29, 31)

}  // namespace swc
