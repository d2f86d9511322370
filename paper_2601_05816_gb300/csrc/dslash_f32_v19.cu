// FP32 hopping-kernel variant 19: variant 18 (32 rhs) with the operands L1-prefetched one direction ahead.
#include "dslash.cuh"

namespace lqcd {
LQCD_DSLASH_VARIANT_NRHS_TU(float, 2, 128, 4, 32, 1)
}  // namespace lqcd
