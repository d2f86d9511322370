// FP32 hopping-kernel variant 16: variant 13 with the operands L1-prefetched two directions ahead.
#include "dslash.cuh"

namespace lqcd {
LQCD_DSLASH_VARIANT_NRHS_TU(float, 2, 128, 4, 16, 2)
}  // namespace lqcd
