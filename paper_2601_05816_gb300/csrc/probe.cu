// Arithmetic-peak probe: the rate at which this GPU retires dependent-chain-free FMAs in
// FP32 or FP64 (SIMT pipes, not tensor cores). The FP64 hopping kernel and the FP64
// Gram-Schmidt are bound by this rate rather than by HBM, so their roofline needs a
// measured denominator.
#include "ctx.h"

namespace lqcd {

// Each thread runs 8 independent FMA chains of `iters` steps; the result is stored so the
// compiler keeps the work. 2 flops per FMA.
template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, T a, T b, T* out) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = x[k] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace lqcd

using namespace lqcd;

extern "C" lqcd_status lqcd_fma_peak(int f64, double* tflops, void* stream) {
  if (tflops == nullptr) return set_error(LQCD_ERR_ARG, "lqcd_fma_peak: null output");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  LQCD_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  LQCD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "attribute");
  const int blocks = sms * 8, threads = 256;
  const int iters = f64 ? 4096 : 65536;
  void* out = nullptr;
  LQCD_CUDA(cudaMalloc(&out, (size_t)blocks * threads * 8), "cudaMalloc(probe)");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  cudaError_t err = cudaSuccess;
  for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {
    cudaEventRecord(e0, s);
    if (f64) fma_probe_kernel<double><<<blocks, threads, 0, s>>>(iters, 0.999999, 1e-7, (double*)out);
    else fma_probe_kernel<float><<<blocks, threads, 0, s>>>(iters, 0.999999f, 1e-7f, (float*)out);
    cudaEventRecord(e1, s);
    err = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;  // the first launch warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return cuda_error(err, "lqcd_fma_peak");
  const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return LQCD_OK;
}
