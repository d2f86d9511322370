// FP32 hopping-kernel variant reading two-row links (LF = 1: FP32 rows, 2: BF16 rows):
// LQCD_DSLASH_VARIANT_LF_TU(rhs per thread, threads, min CTAs/SM, persistent, fixed rhs count, prefetch, LF).
#include "dslash.cuh"

namespace lqcd {
LQCD_DSLASH_VARIANT_LF_TU(2, 128, 4, false, 0, 0, 1)
}  // namespace lqcd
