// Streaming Gram-Schmidt pass, BF16 basis (FP32 arithmetic, FP32 w).
#include "gs_stream_impl.cuh"

namespace lqcd {
cudaError_t launch_gs_stream_bf16(const BlasPlan& plan, int64_t n, int nvec, const void* basis,
                                  int64_t vstride, void* w, const void* coef, bool update, bool dots, bool norm,
                                  void* partials, const int* skip, cudaStream_t stream, const double* oscale,
                                  void* wout, int* blocks_used) {
  return gss::launch_stream<__nv_bfloat162>(plan, n, nvec, basis, vstride, w, coef, update, dots, norm, partials,
                                            skip, stream, oscale, wout, blocks_used);
}
bool gs_stream_passes_supported_bf16(const BlasPlan& plan, int64_t n, int nvec_max) {
  return gss::passes_supported<__nv_bfloat162>(plan, n, nvec_max);
}
}  // namespace lqcd
