// Pipelined FP32 hopping kernel (dslash_pipe.cuh) for 16 rhs: 128 threads with two stages at four CTAs
// per SM or three stages at two, and 256 threads with two stages at two.
#include "dslash_pipe.cuh"

namespace lqcd {
LQCD_DSLASH_PIPE_TU(16, 128, 4, 2)
LQCD_DSLASH_PIPE_TU(16, 128, 2, 3)
LQCD_DSLASH_PIPE_TU(16, 256, 2, 2)
}  // namespace lqcd
