// FP32 hopping-kernel variant 3: 1 rhs per thread, 128 threads per CTA, >= 6 CTA(s) per SM.
#include "dslash.cuh"

namespace lqcd {
LQCD_DSLASH_VARIANT_TU(float, 1, 128, 6, false, false)
}  // namespace lqcd
