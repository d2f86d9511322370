// FP32 hopping-kernel variant 21: variant 20 (64 rhs) with the operands L1-prefetched one direction ahead.
#include "dslash.cuh"

namespace lqcd {
LQCD_DSLASH_VARIANT_NRHS_TU(float, 2, 128, 4, 64, 1)
}  // namespace lqcd
