// FP32 hopping-kernel variant 11: 2 rhs per thread, 256 threads per CTA, >= 2 CTA(s) per SM, persistent CTAs over contiguous site chunks.
#include "dslash.cuh"

namespace lqcd {
LQCD_DSLASH_VARIANT_TU(float, 2, 256, 2, false, true)
}  // namespace lqcd
