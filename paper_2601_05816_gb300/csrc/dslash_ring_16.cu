// FP32 bulk-copy ring hopping kernel (dslash_ring.cuh), 16 rhs.
#include "dslash_ring.cuh"

namespace lqcd {
LQCD_DSLASH_RING_TU(16)
}  // namespace lqcd
