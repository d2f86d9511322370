// FP32 hopping-kernel variant 17: variant 14 (256 threads, >= 2 CTAs/SM, 16 rhs) with the operands L1-prefetched one direction ahead.
#include "dslash.cuh"

namespace lqcd {
LQCD_DSLASH_VARIANT_NRHS_TU(float, 2, 256, 2, 16, 1)
}  // namespace lqcd
