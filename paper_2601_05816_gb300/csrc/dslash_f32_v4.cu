// FP32 hopping-kernel variant 4: 1 rhs per thread, 256 threads per CTA, >= 1 CTA(s) per SM.
#include "dslash.cuh"

namespace lqcd {
LQCD_DSLASH_VARIANT_TU(float, 1, 256, 1, false, false)
}  // namespace lqcd
