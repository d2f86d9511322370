// Extra link and site-block copies built from the structure-of-arrays FP32 copies after
// set-up:
// * site-major copies for the bulk-copy ring hopping kernel (dslash_ring.cuh): one bulk
//   copy moves one link (its 9 complex entries, padded to 80 bytes) or one site's
//   72-real block, so each must be one contiguous, 16-byte aligned run;
// * two-row ("12-real") link copies, rows 0 and 1 of each SU(3) link in FP32 and in
//   BF16, for the kernels that rebuild the third row.
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

// rows 0 and 1 of each link ([4][9][V] entries 0..5 of each mu) rounded to BF16 pairs
__global__ void links_r12_bf16_kernel(int V, const float2* __restrict__ l32, __nv_bfloat162* __restrict__ out) {
  const int64_t total = (int64_t)4 * 6 * V;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t mu = q / (6 * (int64_t)V), rest = q % (6 * (int64_t)V);
    out[q] = __float22bfloat162_rn(l32[mu * 9 * V + rest]);
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

cudaError_t launch_links_r12(int V, const void* links32, void* r12, void* r12_bf16, cudaStream_t s) {
  // FP32 rows: entries 0..5 of each direction are contiguous in the [4][9][V] layout
  for (int mu = 0; mu < 4; ++mu) {
    cudaError_t e = cudaMemcpyAsync((float2*)r12 + (int64_t)mu * 6 * V, (const float2*)links32 + (int64_t)mu * 9 * V,
                                    sizeof(float2) * 6 * (size_t)V, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  links_r12_bf16_kernel<<<grid_of((int64_t)24 * V), 256, 0, s>>>(V, (const float2*)links32, (__nv_bfloat162*)r12_bf16);
  return cudaGetLastError();
}

cudaError_t launch_blocks_aos(int V, const void* blk32, void* aos, cudaStream_t s) {
  blocks_aos_kernel<<<grid_of((int64_t)18 * V), 256, 0, s>>>(V, (const float4*)blk32, (float4*)aos);
  return cudaGetLastError();
}

}  // namespace lqcd
