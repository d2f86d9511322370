// FP32 hopping-kernel variant 10: 2 rhs per thread, 128 threads per CTA, >= 4 CTA(s) per SM, batched loads, persistent CTAs over contiguous site chunks.
#include "dslash.cuh"

namespace lqcd {
LQCD_DSLASH_VARIANT_TU(float, 2, 128, 4, true, true)
}  // namespace lqcd
