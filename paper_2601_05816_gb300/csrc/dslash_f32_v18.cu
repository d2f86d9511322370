// FP32 hopping-kernel variant 18: 2 rhs per thread, 128 threads, >= 4 CTAs/SM, compiled for 32 rhs.
#include "dslash.cuh"

namespace lqcd {
LQCD_DSLASH_VARIANT_NRHS_TU(float, 2, 128, 4, 32, 0)
}  // namespace lqcd
