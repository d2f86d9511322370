// FP64 hopping-kernel variant 1: 1 rhs per thread, 128 threads per CTA, >= 4 CTA(s) per SM.
#include "dslash.cuh"

namespace lqcd {
LQCD_DSLASH_VARIANT_TU(double, 1, 128, 4, false, false)
}  // namespace lqcd
