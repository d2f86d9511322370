// Site-major FP32 copies of the links and site blocks for the bulk-copy ring hopping
// kernel (dslash_ring.cuh): one bulk copy moves one link (its 9 complex entries,
// padded to 80 bytes) or one site's 72-real block, so each must be one contiguous,
// 16-byte aligned run. Built from the structure-of-arrays copies after set-up.
#include "kernels.h"

namespace lqcd {

// links [4][9][V] float2 (entry-major) -> [4][V][10] float2 (link-major, 10th entry 0)
__global__ void links_aos_kernel(int V, const float2* __restrict__ soa, float2* __restrict__ aos) {
  const int64_t total = (int64_t)4 * V * 10;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(q % 10);
    const int64_t l = q / 10;        // mu * V + site
    const int mu = (int)(l / V), site = (int)(l % V);
    aos[q] = e < 9 ? soa[((int64_t)mu * 9 + e) * V + site] : make_float2(0.f, 0.f);
  }
}

// blocks [18][V] float4 (16-byte chunk-major) -> [V][18] float4 (site-major)
__global__ void blocks_aos_kernel(int V, const float4* __restrict__ soa, float4* __restrict__ aos) {
  const int64_t total = (int64_t)18 * V;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(q % 18);
    const int64_t site = q / 18;
    aos[q] = soa[(int64_t)k * V + site];
  }
}

static int grid_of(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (int)(b > 65535 * 8 ? 65535 * 8 : (b < 1 ? 1 : b));
}

cudaError_t launch_links_aos(int V, const void* links32, void* aos, cudaStream_t s) {
  links_aos_kernel<<<grid_of((int64_t)40 * V), 256, 0, s>>>(V, (const float2*)links32, (float2*)aos);
  return cudaGetLastError();
}

cudaError_t launch_blocks_aos(int V, const void* blk32, void* aos, cudaStream_t s) {
  blocks_aos_kernel<<<grid_of((int64_t)18 * V), 256, 0, s>>>(V, (const float4*)blk32, (float4*)aos);
  return cudaGetLastError();
}

}  // namespace lqcd
