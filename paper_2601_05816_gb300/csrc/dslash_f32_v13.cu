// FP32 hopping-kernel variant 13: variant 1 (2 rhs per thread, 128 threads, >= 4 CTAs/SM) compiled for 16 rhs.
#include "dslash.cuh"

namespace lqcd {
LQCD_DSLASH_VARIANT_NRHS_TU(float, 2, 128, 4, 16, 0)
}  // namespace lqcd
