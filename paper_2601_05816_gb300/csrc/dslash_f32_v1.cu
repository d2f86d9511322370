// FP32 hopping-kernel variant 1: 2 rhs per thread, 128 threads per CTA, >= 4 CTA(s) per SM.
#include "dslash.cuh"

namespace lqcd {
LQCD_DSLASH_VARIANT_TU(float, 2, 128, 4, false, false)
}  // namespace lqcd
