// FP32 hopping-kernel variant 10: 2 rhs per thread, 128 threads per CTA, >= 3 CTA(s) per SM, batched loads.
#include "dslash.cuh"

namespace lqcd {
LQCD_DSLASH_VARIANT_TU(float, 2, 128, 3, true)
}  // namespace lqcd
