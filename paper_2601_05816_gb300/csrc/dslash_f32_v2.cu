// FP32 hopping-kernel variant 2: 1 rhs per thread, 128 threads per CTA, >= 1 CTA(s) per SM.
#include "dslash.cuh"

namespace lqcd {
LQCD_DSLASH_VARIANT_TU(float, 1, 128, 1, false, false)
}  // namespace lqcd
