// Hopping kernel on BF16-stored spinors with FP32 arithmetic: the operator applied to a
// BF16 basis vector of the mixed-precision solver (with the context's BF16 two-row links
// when that link storage is chosen). Pass A and the full operator read
// a BF16 hop input (and self input); pass B reads the FP32 intermediate as hop input
// and the BF16 vector as self input.
#include "dslash.cuh"

namespace lqcd {

using bf2 = __nv_bfloat162;

cudaError_t launch_dslash_bf16(const DslashArgs<float>& a, int self_mode, int post_mode, bool hop_bf16,
                               cudaStream_t s) {
  if (a.link_format == 2) {  // BF16 two-row links as well
    if (a.lay.nrhs % 2 == 0 && a.lay.nrhs / 2 <= 128) {
      if (hop_bf16) return launch_dslash_variant<float, 2, 128, 4, false, false, bf2, bf2, 0, 0, 2>(a, self_mode, post_mode, s);
      return launch_dslash_variant<float, 2, 128, 4, false, false, float2, bf2, 0, 0, 2>(a, self_mode, post_mode, s);
    }
    if (a.lay.nrhs <= 128) {
      if (hop_bf16) return launch_dslash_variant<float, 1, 128, 6, false, false, bf2, bf2, 0, 0, 2>(a, self_mode, post_mode, s);
      return launch_dslash_variant<float, 1, 128, 6, false, false, float2, bf2, 0, 0, 2>(a, self_mode, post_mode, s);
    }
    return cudaErrorInvalidValue;
  }
  if (a.lay.nrhs % 2 == 0 && a.lay.nrhs / 2 <= 128) {
    if (hop_bf16) return launch_dslash_variant<float, 2, 128, 4, false, false, bf2, bf2>(a, self_mode, post_mode, s);
    return launch_dslash_variant<float, 2, 128, 4, false, false, float2, bf2>(a, self_mode, post_mode, s);
  }
  if (a.lay.nrhs <= 128) {
    if (hop_bf16) return launch_dslash_variant<float, 1, 128, 6, false, false, bf2, bf2>(a, self_mode, post_mode, s);
    return launch_dslash_variant<float, 1, 128, 6, false, false, float2, bf2>(a, self_mode, post_mode, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lqcd
