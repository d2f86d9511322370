// Layout conversion kernels: canonical <-> packed spinor blocks, gauge-field packing.
//
// The paper keeps psi as one vector per rhs (column-major block, Eq. (1)) and
// notes that reordering before and after a solve costs little (Sec. III-A-2);
// these kernels are that reordering. Packed spinors put the rhs innermost
// (Eq. (2) row-major), sites in eo order; packed links are
// [mu][entry][site] structure-of-arrays so that consecutive sites read
// consecutive addresses, with the fermion time boundary factor folded into
// U_0 on the last time slice (so the hopping kernel needs no boundary branch).
#include "kernels.h"

namespace lqcd {

// Decode a packed element index into (site i, component c, rhs r).
__device__ __forceinline__ void decode_packed(int64_t e, int nrhs, int log_s, int64_t& i, int& c, int& r) {
  r = (int)(e % nrhs);
  int64_t q = e / nrhs;
  const int64_t S = int64_t(1) << log_s;
  const int64_t s_in = q & (S - 1);
  q >>= log_s;
  c = (int)(q % 12);
  const int64_t tile = q / 12;
  i = (tile << log_s) + s_in;
}

// Canonical site index (within the canonical block) of packed site i.
__device__ __forceinline__ int64_t canonical_site(const Geom& g, int sites, int64_t i) {
  if (sites == 0) {  // full: packed eo index -> site number
    const int p = i >= g.Vh ? 1 : 0;
    const int cb = (int)(i - p * g.Vh);
    return site_coords(g, p, cb).lex;
  }
  return i;  // one parity: canonical order is cb order
}

__device__ __forceinline__ float2 cvt(__nv_bfloat162 v, float2*) { return __bfloat1622float2(v); }
__device__ __forceinline__ __nv_bfloat162 cvt(float2 v, __nv_bfloat162*) { return __float22bfloat162_rn(v); }
template <typename C>
__device__ __forceinline__ C cvt(C v, C*) { return v; }

// Canonical <-> packed; CIN/COUT differ for the BF16 packed storage (complex64 canonical).
template <typename CIN, typename COUT, bool TO_PACKED>
__global__ void spinor_layout_kernel(Geom g, int sites, int nrhs, int log_s, int64_t n_sites,
                                     const CIN* __restrict__ in, COUT* __restrict__ out) {
  const int64_t total = n_sites * 12 * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i; int c, r;
    decode_packed(e, nrhs, log_s, i, c, r);
    const int64_t cs = canonical_site(g, sites, i);
    const int64_t ce = ((int64_t)r * n_sites + cs) * 12 + c;
    if (TO_PACKED) out[e] = cvt(in[ce], (COUT*)nullptr);
    else out[ce] = cvt(in[e], (COUT*)nullptr);
  }
}

cudaError_t launch_spinor_layout(const Geom& g, int sites, int nrhs, int log_s, bool to_packed,
                                 bool f64, const void* in, void* out, cudaStream_t stream, bool bf16) {
  const int64_t n_sites = sites == 0 ? g.V : g.Vh;
  const int64_t total = n_sites * 12 * nrhs;
  const int threads = 256;
  int64_t blocks64 = (total + threads - 1) / threads;
  const int blocks = (int)(blocks64 > 65535 * 16 ? 65535 * 16 : blocks64);
  using bf2 = __nv_bfloat162;
  if (bf16) {
    if (to_packed)
      spinor_layout_kernel<float2, bf2, true><<<blocks, threads, 0, stream>>>(
          g, sites, nrhs, log_s, n_sites, (const float2*)in, (bf2*)out);
    else
      spinor_layout_kernel<bf2, float2, false><<<blocks, threads, 0, stream>>>(
          g, sites, nrhs, log_s, n_sites, (const bf2*)in, (float2*)out);
  } else if (f64) {
    if (to_packed)
      spinor_layout_kernel<double2, double2, true><<<blocks, threads, 0, stream>>>(
          g, sites, nrhs, log_s, n_sites, (const double2*)in, (double2*)out);
    else
      spinor_layout_kernel<double2, double2, false><<<blocks, threads, 0, stream>>>(
          g, sites, nrhs, log_s, n_sites, (const double2*)in, (double2*)out);
  } else {
    if (to_packed)
      spinor_layout_kernel<float2, float2, true><<<blocks, threads, 0, stream>>>(
          g, sites, nrhs, log_s, n_sites, (const float2*)in, (float2*)out);
    else
      spinor_layout_kernel<float2, float2, false><<<blocks, threads, 0, stream>>>(
          g, sites, nrhs, log_s, n_sites, (const float2*)in, (float2*)out);
  }
  return cudaGetLastError();
}

// Column repacking between two FP64 packed blocks of the same sites with different
// rhs counts (the solver's compaction of its active rhs): gather
//   dst(layout nd)[i][c][k] = src(layout ns)[i][c][map[k]],  k < nd,
// or scatter
//   dst(layout nd)[i][c][map[k]] = src(layout ns)[i][c][k],  k < ns.
__global__ void repack_columns_kernel(int64_t n_sites, PackedLayout ls, PackedLayout ld, ColumnMap map,
                                      bool scatter, const double2* __restrict__ src, double2* __restrict__ dst) {
  const int nk = scatter ? ls.nrhs : ld.nrhs;
  const int64_t total = n_sites * 12 * nk;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % nk);
    const int64_t q = e / nk;
    const int c = (int)(q % 12);
    const int64_t i = q / 12;
    if (scatter) dst[ld.index(i, c, map.col[k])] = src[ls.index(i, c, k)];
    else dst[ld.index(i, c, k)] = src[ls.index(i, c, map.col[k])];
  }
}

cudaError_t launch_repack_columns(int64_t n_sites, PackedLayout ls, PackedLayout ld, const ColumnMap& map,
                                  bool scatter, const void* src, void* dst, cudaStream_t stream) {
  const int nk = scatter ? ls.nrhs : ld.nrhs;
  const int64_t total = n_sites * 12 * nk;
  const int threads = 256;
  const int64_t b = (total + threads - 1) / threads;
  const int blocks = (int)(b > 65535 * 16 ? 65535 * 16 : (b < 1 ? 1 : b));
  repack_columns_kernel<<<blocks, threads, 0, stream>>>(n_sites, ls, ld, map, scatter, (const double2*)src,
                                                        (double2*)dst);
  return cudaGetLastError();
}

// Canonical U [V][4][3][3] complex128 -> packed [4][9][V] in FP64 and FP32, eo site order.
__global__ void gauge_pack_kernel(Geom g, int time_bc, const double2* __restrict__ U,
                                  double2* __restrict__ l64, float2* __restrict__ l32) {
  const int64_t total = (int64_t)36 * g.V;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % g.V);
    const int me = (int)(e / g.V);  // mu * 9 + entry
    const int mu = me / 9, ent = me % 9;
    const int p = i >= g.Vh ? 1 : 0;
    const Coord c = site_coords(g, p, i - p * g.Vh);
    double2 u = U[((int64_t)c.lex * 4 + mu) * 9 + ent];
    if (mu == 0 && c.t == g.T - 1 && time_bc != 1) { u.x *= time_bc; u.y *= time_bc; }
    l64[e] = u;
    l32[e] = make_float2((float)u.x, (float)u.y);
  }
}

cudaError_t launch_gauge_pack(const Geom& g, int time_bc, const void* U, void* l64, void* l32,
                              cudaStream_t stream) {
  const int64_t total = (int64_t)36 * g.V;
  const int threads = 256;
  int64_t b = (total + threads - 1) / threads;
  const int blocks = (int)(b > 65535 * 16 ? 65535 * 16 : b);
  gauge_pack_kernel<<<blocks, threads, 0, stream>>>(g, time_bc, (const double2*)U, (double2*)l64,
                                                     (float2*)l32);
  return cudaGetLastError();
}

}  // namespace lqcd
