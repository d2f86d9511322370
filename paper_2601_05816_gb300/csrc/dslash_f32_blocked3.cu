// FP32 hopping-kernel variant with the blocked site mapping and the x, y, z, t direction order:
// LQCD_DSLASH_VARIANT_ORD_TU(rhs per thread, threads, min CTAs/SM, fixed rhs count, prefetch distance).
#include "dslash.cuh"

namespace lqcd {
LQCD_DSLASH_VARIANT_ORD_TU(2, 256, 2, 16, 2)
}  // namespace lqcd
