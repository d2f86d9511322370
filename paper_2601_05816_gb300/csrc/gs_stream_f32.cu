// Streaming Gram-Schmidt pass, FP32 basis.
#include "gs_stream_impl.cuh"

namespace lqcd {
cudaError_t launch_gs_stream_f32(const BlasPlan& plan, int64_t n, int nvec, const void* basis, int64_t vstride,
                                 void* w, const void* coef, bool update, bool dots, bool norm, void* partials,
                                 const int* skip, cudaStream_t stream, const double* oscale, void* wout,
                                 int* blocks_used) {
  return gss::launch_stream<float2>(plan, n, nvec, basis, vstride, w, coef, update, dots, norm, partials, skip,
                                    stream, oscale, wout, blocks_used);
}
bool gs_stream_passes_supported_f32(const BlasPlan& plan, int64_t n, int nvec_max) {
  return gss::passes_supported<float2>(plan, n, nvec_max);
}
}  // namespace lqcd
