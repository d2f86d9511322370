// FP64 hopping-kernel variant 4: cp.async pipeline of 2 stages, 1 rhs per thread, 128 threads per CTA.
#include "dslash_async.cuh"

namespace lqcd {
LQCD_DSLASH_ASYNC_VARIANT_TU(double, 1, 128, 1, 2)
}  // namespace lqcd
