// FP32 hopping-kernel variant 6: cp.async pipeline of 2 stages, 2 rhs per thread, 128 threads per CTA.
#include "dslash_async.cuh"

namespace lqcd {
LQCD_DSLASH_ASYNC_VARIANT_TU(float, 2, 128, 1, 2)
}  // namespace lqcd
