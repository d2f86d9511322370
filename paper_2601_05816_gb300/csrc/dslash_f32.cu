// FP32 (complex64) instantiations of the multi-rhs hopping kernel.
#include "dslash.cuh"
#include "kernels.h"

namespace lqcd {

template <int NR>
static cudaError_t launch_nr(const DslashArgs<float>& a, int self_mode, int post_mode, cudaStream_t s) {
  const int G = a.lay.nrhs / NR;
  dim3 block(G, G >= 128 ? 1 : 128 / G);
  dim3 grid((a.n_target + block.y - 1) / block.y);
#define DS(SM, PM) dslash_kernel<float, NR, SM, PM><<<grid, block, 0, s>>>(a)
  if (self_mode == SELF_SCALAR && post_mode == POST_NONE) DS(SELF_SCALAR, POST_NONE);
  else if (self_mode == SELF_BLOCK && post_mode == POST_NONE) DS(SELF_BLOCK, POST_NONE);
  else if (self_mode == SELF_NONE && post_mode == POST_SCALAR) DS(SELF_NONE, POST_SCALAR);
  else if (self_mode == SELF_NONE && post_mode == POST_BLOCKINV) DS(SELF_NONE, POST_BLOCKINV);
  else if (self_mode == SELF_SCALAR && post_mode == POST_SCALAR) DS(SELF_SCALAR, POST_SCALAR);
  else if (self_mode == SELF_SCALAR && post_mode == POST_BLOCKINV) DS(SELF_SCALAR, POST_BLOCKINV);
  else return cudaErrorInvalidValue;
#undef DS
  return cudaGetLastError();
}

template <>
cudaError_t launch_dslash<float>(const DslashArgs<float>& a, int self_mode, int post_mode, int nr,
                                 cudaStream_t stream) {
  if (nr == 2) return launch_nr<2>(a, self_mode, post_mode, stream);
  return launch_nr<1>(a, self_mode, post_mode, stream);
}

}  // namespace lqcd
