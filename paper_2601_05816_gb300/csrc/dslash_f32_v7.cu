// FP32 hopping-kernel variant 7: 2 rhs per thread, 128 threads per CTA, >= 4 CTA(s) per SM, batched loads.
#include "dslash.cuh"

namespace lqcd {
LQCD_DSLASH_VARIANT_TU(float, 2, 128, 4, true, false)
}  // namespace lqcd
