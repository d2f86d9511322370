// Software-pipelined variant of the multi-rhs hopping kernel.
//
// Same arithmetic as dslash_kernel (dslash.cuh), but every operand of the eight
// hopping directions moves through shared memory with cp.async: while the
// thread computes direction d, the copies of directions d+1 .. d+STAGES-1 are in
// flight, so the neighbour spinors and links of several directions are
// outstanding per thread without occupying registers. Per thread and stage the
// buffer holds the 12 spin-colour components of its NR rhs; per site and stage
// one lane (threadIdx.x == 0) copies the 3x3 link, which the site's lanes then
// read after a barrier. The self-term input of pass B / the full operator is a
// ninth pipeline item, and the site block (A or A^{-1}) is copied with the first
// stage. Copies of sites past the end are skipped but those threads still take
// part in the barriers.
#pragma once
#include "dslash.cuh"

namespace lqcd {

template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem_dst, const void* gsrc) {
  const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(dst), "l"(gsrc), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Bytes of NR consecutive complex numbers.
template <typename Real, int NR> struct VecBytes { static constexpr int value = (int)sizeof(Real) * 2 * NR; };

template <typename Real, int NR>
__device__ __forceinline__ void mc_from_smem(MC<Real, NR>& a, const unsigned char* p) {
  const Real* q = reinterpret_cast<const Real*>(p);
#pragma unroll
  for (int k = 0; k < NR; ++k) { a.re[k] = q[2 * k]; a.im[k] = q[2 * k + 1]; }
}

template <typename Real>
__host__ __device__ constexpr int block_chunk_count() { return 72 * (int)sizeof(Real) / 16; }

// Shared memory of one CTA (nthr threads, sy sites): spinor stages, link stages
// (rounded up to 16 bytes), site blocks.
template <typename Real, int STAGES>
__host__ __device__ constexpr size_t dslash_async_link_bytes(int sy) {
  return ((size_t)STAGES * sy * 9 * sizeof(typename Cplx<Real>::T) + 15) / 16 * 16;
}
template <typename Real, int NR, int STAGES>
__host__ __device__ constexpr size_t dslash_async_smem(int nthr, int sy) {
  return (size_t)STAGES * 12 * nthr * VecBytes<Real, NR>::value + dslash_async_link_bytes<Real, STAGES>(sy) +
         (size_t)sy * 72 * sizeof(Real);
}

template <typename Real, int NR, int MU, int DIR>
__device__ __forceinline__ void hop_from_smem(const unsigned char* sp_stage, const typename Cplx<Real>::T* sl_site,
                                              int nthr, int tid, MC<Real, NR> acc[12]) {
  using C = typename Cplx<Real>::T;
  constexpr int VB = VecBytes<Real, NR>::value;
  C u[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) u[e] = sl_site[e];
  MC<Real, NR> up[6], dn[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    mc_from_smem<Real, NR>(up[k], sp_stage + ((size_t)k * nthr + tid) * VB);
    mc_from_smem<Real, NR>(dn[k], sp_stage + ((size_t)(6 + k) * nthr + tid) * VB);
  }
  hop_compute<Real, NR, MU, DIR>(u, up, dn, acc);
}

template <typename Real, int NR, int SELF, int POST, int MAXT, int MINB, int STAGES>
__global__ void __launch_bounds__(MAXT, MINB) dslash_async_kernel(DslashArgs<Real> a) {
  using C = typename Cplx<Real>::T;
  constexpr int VB = VecBytes<Real, NR>::value;
  constexpr int NITEMS = SELF != SELF_NONE ? 9 : 8;
  extern __shared__ __align__(16) unsigned char smem[];
  if (a.skip != nullptr && *a.skip != 0) return;
  const int nthr = blockDim.x * blockDim.y;
  const int sy = blockDim.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  unsigned char* sp = smem;
  C* sl = reinterpret_cast<C*>(smem + (size_t)STAGES * 12 * nthr * VB);
  Real* sb = reinterpret_cast<Real*>(reinterpret_cast<unsigned char*>(sl) + dslash_async_link_bytes<Real, STAGES>(sy));

  const int site = blockIdx.x * sy + threadIdx.y;
  const bool active = site < a.n_target;
  const int r0 = threadIdx.x * NR;
  int p, cb;
  if (a.full) {
    p = (active && site >= a.g.Vh) ? 1 : 0;
    cb = active ? site - p * a.g.Vh : 0;
  } else {
    p = a.target_parity;
    cb = active ? site : 0;
  }
  const int eo_site = p * a.g.Vh + cb;
  const C* hin = a.full ? a.hop_in + (1 - p) * a.half_elems : a.hop_in;
  const int64_t base = a.full ? p * a.half_elems : 0;

  // neighbour cb index and link site of the eight directions (order t+, t-, z+, z-, y+, y-, x+, x-)
  int ncb[8], lsite[8];
  {
    const Coord c = site_coords(a.g, p, cb);
    const int here = p * a.g.Vh + cb;
    int nl;
    nl = neighbour_lex<0, +1>(a.g, c); ncb[0] = nl >> 1; lsite[0] = here;
    nl = neighbour_lex<0, -1>(a.g, c); ncb[1] = nl >> 1; lsite[1] = (1 - p) * a.g.Vh + ncb[1];
    nl = neighbour_lex<1, +1>(a.g, c); ncb[2] = nl >> 1; lsite[2] = here;
    nl = neighbour_lex<1, -1>(a.g, c); ncb[3] = nl >> 1; lsite[3] = (1 - p) * a.g.Vh + ncb[3];
    nl = neighbour_lex<2, +1>(a.g, c); ncb[4] = nl >> 1; lsite[4] = here;
    nl = neighbour_lex<2, -1>(a.g, c); ncb[5] = nl >> 1; lsite[5] = (1 - p) * a.g.Vh + ncb[5];
    nl = neighbour_lex<3, +1>(a.g, c); ncb[6] = nl >> 1; lsite[6] = here;
    nl = neighbour_lex<3, -1>(a.g, c); ncb[7] = nl >> 1; lsite[7] = (1 - p) * a.g.Vh + ncb[7];
  }

  auto issue = [&](int item) {
    if (active && item < NITEMS) {
      unsigned char* st = sp + (size_t)(item % STAGES) * 12 * nthr * VB;
      if (item < 8) {
#pragma unroll
        for (int k = 0; k < 12; ++k) cp_async<VB>(st + ((size_t)k * nthr + tid) * VB, hin + a.lay.index(ncb[item], k, r0));
        if (threadIdx.x == 0) {
          C* dst = sl + ((size_t)(item % STAGES) * sy + threadIdx.y) * 9;
          const C* src = a.links + (int64_t)((item >> 1) * 9) * a.g.V + lsite[item];
#pragma unroll
          for (int e = 0; e < 9; ++e) cp_async<(int)sizeof(C)>(dst + e, src + (int64_t)e * a.g.V);
        }
      } else {
        const C* src = a.self_in + base;
#pragma unroll
        for (int k = 0; k < 12; ++k) cp_async<VB>(st + ((size_t)k * nthr + tid) * VB, src + a.lay.index(cb, k, r0));
      }
    }
    cp_commit();
  };

  // the site block (A for SELF_BLOCK, A^{-1} for POST_BLOCKINV) rides with the first stage
  if ((SELF == SELF_BLOCK || POST == POST_BLOCKINV) && active && threadIdx.x == 0) {
    const Real* blk = POST == POST_BLOCKINV ? a.blocks_inv : a.blocks;
    constexpr int NCH = block_chunk_count<Real>();
#pragma unroll
    for (int q = 0; q < NCH; ++q)
      cp_async<16>(reinterpret_cast<unsigned char*>(sb + threadIdx.y * 72) + 16 * q,
                   reinterpret_cast<const unsigned char*>(blk) + ((size_t)q * a.g.V + eo_site) * 16);
  }
#pragma unroll
  for (int s = 0; s < STAGES - 1; ++s) issue(s);

  MC<Real, NR> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) mc_zero(acc[k]);
  MC<Real, NR> self[12];

#pragma unroll
  for (int item = 0; item < NITEMS; ++item) {
    issue(item + STAGES - 1);
    cp_wait<STAGES - 1>();
    __syncthreads();
    const unsigned char* st = sp + (size_t)(item % STAGES) * 12 * nthr * VB;
    const C* ls = sl + ((size_t)(item % STAGES) * sy + threadIdx.y) * 9;
    if (active) {
      switch (item) {
        case 0: hop_from_smem<Real, NR, 0, +1>(st, ls, nthr, tid, acc); break;
        case 1: hop_from_smem<Real, NR, 0, -1>(st, ls, nthr, tid, acc); break;
        case 2: hop_from_smem<Real, NR, 1, +1>(st, ls, nthr, tid, acc); break;
        case 3: hop_from_smem<Real, NR, 1, -1>(st, ls, nthr, tid, acc); break;
        case 4: hop_from_smem<Real, NR, 2, +1>(st, ls, nthr, tid, acc); break;
        case 5: hop_from_smem<Real, NR, 2, -1>(st, ls, nthr, tid, acc); break;
        case 6: hop_from_smem<Real, NR, 3, +1>(st, ls, nthr, tid, acc); break;
        case 7: hop_from_smem<Real, NR, 3, -1>(st, ls, nthr, tid, acc); break;
        default:
#pragma unroll
          for (int k = 0; k < 12; ++k) mc_from_smem<Real, NR>(self[k], st + ((size_t)k * nthr + tid) * VB);
      }
    }
    __syncthreads();
  }
  cp_wait<0>();
  if (!active) return;

#pragma unroll
  for (int k = 0; k < 12; ++k)
#pragma unroll
    for (int q = 0; q < NR; ++q) { acc[k].re[q] *= a.c_hop; acc[k].im[q] *= a.c_hop; }
  const Real* bl = sb + threadIdx.y * 72;
  if (SELF == SELF_SCALAR) {
#pragma unroll
    for (int k = 0; k < 12; ++k)
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        acc[k].re[q] = fma(a.self_scalar, self[k].re[q], acc[k].re[q]);
        acc[k].im[q] = fma(a.self_scalar, self[k].im[q], acc[k].im[q]);
      }
  } else if (SELF == SELF_BLOCK) {
    MC<Real, NR> t[12];
    block_matvec<Real, NR>(bl, self, t);
    block_matvec<Real, NR>(bl + 36, self + 6, t + 6);
#pragma unroll
    for (int k = 0; k < 12; ++k)
#pragma unroll
      for (int q = 0; q < NR; ++q) { acc[k].re[q] += t[k].re[q]; acc[k].im[q] += t[k].im[q]; }
  }
  C* op = a.out + base;
  if (POST == POST_BLOCKINV) {
    MC<Real, NR> t[12];
    block_matvec<Real, NR>(bl, acc, t);
    block_matvec<Real, NR>(bl + 36, acc + 6, t + 6);
#pragma unroll
    for (int k = 0; k < 12; ++k) mc_store(op + a.lay.index(cb, k, r0), t[k]);
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      if (POST == POST_SCALAR) {
#pragma unroll
        for (int q = 0; q < NR; ++q) { acc[k].re[q] *= a.post_scalar; acc[k].im[q] *= a.post_scalar; }
      }
      mc_store(op + a.lay.index(cb, k, r0), acc[k]);
    }
  }
}

template <typename Real, int NR, int MAXT, int MINB, int STAGES, int SM, int PM>
static cudaError_t launch_async_one(const DslashArgs<Real>& a, dim3 grid, dim3 block, cudaStream_t s) {
  auto kern = dslash_async_kernel<Real, NR, SM, PM, MAXT, MINB, STAGES>;
  const size_t smem = dslash_async_smem<Real, NR, STAGES>(block.x * block.y, block.y);
  // the opt-in shared-memory size is raised whenever a launch shape needs more
  // than this instantiation was configured for (benign race: the attribute only grows)
  static size_t configured = 0;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  kern<<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename Real, int NR, int MAXT, int MINB, int STAGES>
cudaError_t launch_dslash_async_variant(const DslashArgs<Real>& a, int self_mode, int post_mode, cudaStream_t s) {
  const int G = a.lay.nrhs / NR;
  dim3 block(G, G >= MAXT ? 1 : MAXT / G);
  dim3 grid((a.n_target + block.y - 1) / block.y);
#define LQCD_DSA(SMODE, PMODE) return launch_async_one<Real, NR, MAXT, MINB, STAGES, SMODE, PMODE>(a, grid, block, s)
  if (self_mode == SELF_SCALAR && post_mode == POST_NONE) LQCD_DSA(SELF_SCALAR, POST_NONE);
  if (self_mode == SELF_BLOCK && post_mode == POST_NONE) LQCD_DSA(SELF_BLOCK, POST_NONE);
  if (self_mode == SELF_NONE && post_mode == POST_SCALAR) LQCD_DSA(SELF_NONE, POST_SCALAR);
  if (self_mode == SELF_NONE && post_mode == POST_BLOCKINV) LQCD_DSA(SELF_NONE, POST_BLOCKINV);
  if (self_mode == SELF_SCALAR && post_mode == POST_SCALAR) LQCD_DSA(SELF_SCALAR, POST_SCALAR);
  if (self_mode == SELF_SCALAR && post_mode == POST_BLOCKINV) LQCD_DSA(SELF_SCALAR, POST_BLOCKINV);
#undef LQCD_DSA
  return cudaErrorInvalidValue;
}

#define LQCD_DSLASH_ASYNC_VARIANT_TU(REAL, NR, MAXT, MINB, STAGES)                                             \
  template cudaError_t launch_dslash_async_variant<REAL, NR, MAXT, MINB, STAGES>(const DslashArgs<REAL>&, int, \
                                                                                 int, cudaStream_t);

}  // namespace lqcd
