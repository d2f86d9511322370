// FP32 hopping-kernel variant 5: 2 rhs per thread, 256 threads per CTA, >= 2 CTA(s) per SM.
#include "dslash.cuh"

namespace lqcd {
LQCD_DSLASH_VARIANT_TU(float, 2, 256, 2, false, false)
}  // namespace lqcd
