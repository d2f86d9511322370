// FP64 hopping-kernel variant 7: 1 rhs per thread, 64 threads per CTA, >= 8 CTA(s) per SM, batched loads.
#include "dslash.cuh"

namespace lqcd {
LQCD_DSLASH_VARIANT_TU(double, 1, 64, 8, true)
}  // namespace lqcd
