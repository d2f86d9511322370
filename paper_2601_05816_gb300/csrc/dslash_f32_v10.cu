// FP32 hopping-kernel variant 10: cp.async pipeline of 3 stages, 1 rhs per thread, 256 threads per CTA.
#include "dslash_async.cuh"

namespace lqcd {
LQCD_DSLASH_ASYNC_VARIANT_TU(float, 1, 256, 1, 3)
}  // namespace lqcd
