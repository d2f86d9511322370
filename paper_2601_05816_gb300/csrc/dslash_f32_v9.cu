// FP32 hopping-kernel variant 9: cp.async pipeline of 4 stages, 1 rhs per thread, 128 threads per CTA.
#include "dslash_async.cuh"

namespace lqcd {
LQCD_DSLASH_ASYNC_VARIANT_TU(float, 1, 128, 1, 4)
}  // namespace lqcd
