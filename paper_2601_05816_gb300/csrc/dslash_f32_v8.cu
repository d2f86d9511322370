// FP32 hopping-kernel variant 8: 2 rhs per thread, 64 threads per CTA, >= 8 CTA(s) per SM, batched loads.
#include "dslash.cuh"

namespace lqcd {
LQCD_DSLASH_VARIANT_TU(float, 2, 64, 8, true, false)
}  // namespace lqcd
