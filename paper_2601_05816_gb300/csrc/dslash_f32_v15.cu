// FP32 hopping-kernel variant 15: variant 13 with the operands L1-prefetched one direction ahead.
#include "dslash.cuh"

namespace lqcd {
LQCD_DSLASH_VARIANT_NRHS_TU(float, 2, 128, 4, 16, 1)
}  // namespace lqcd
