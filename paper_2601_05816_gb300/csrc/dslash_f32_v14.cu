// FP32 hopping-kernel variant 14: variant 5 (2 rhs per thread, 256 threads, >= 2 CTAs/SM) compiled for 16 rhs.
#include "dslash.cuh"

namespace lqcd {
LQCD_DSLASH_VARIANT_NRHS_TU(float, 2, 256, 2, 16, 0)
}  // namespace lqcd
