// pa_f32_r9.cu -- single-precision innermost passes of length 9 * 2^lg (smooth transform lengths).
#include "pa_launch.cuh"

namespace pa {
PA_INSTANTIATE_ODD(float, 9)
}  // namespace pa
