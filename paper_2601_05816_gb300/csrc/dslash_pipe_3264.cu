// Pipelined FP32 hopping kernel (dslash_pipe.cuh) for 32 and 64 rhs: 128 threads, two stages.
#include "dslash_pipe.cuh"

namespace lqcd {
LQCD_DSLASH_PIPE_TU(32, 128, 4, 2)
LQCD_DSLASH_PIPE_TU(64, 128, 4, 2)
}  // namespace lqcd
