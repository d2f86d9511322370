// FP32 hopping-kernel variant 7: cp.async pipeline of 3 stages, 2 rhs per thread, 128 threads per CTA.
#include "dslash_async.cuh"

namespace lqcd {
LQCD_DSLASH_ASYNC_VARIANT_TU(float, 2, 128, 1, 3)
}  // namespace lqcd
