// pa_f64_r3.cu -- double-precision innermost passes of length 3 * 2^lg (smooth transform lengths).
#include "pa_launch.cuh"

namespace pa {
PA_INSTANTIATE_ODD(double, 3)
}  // namespace pa
