// FP32 bulk-copy ring hopping kernel (dslash_ring.cuh), 32 rhs.
#include "dslash_ring.cuh"

namespace lqcd {
LQCD_DSLASH_RING_TU(32)
}  // namespace lqcd
