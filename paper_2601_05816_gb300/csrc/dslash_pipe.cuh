// Pipelined FP32 hopping kernel for a rhs count fixed at compile time (16, 32 or 64).
//
// The arithmetic is that of dslash_kernel (Sec. III-A-1: spin projection, SU(3) multiply
// and reconstruction per direction, the clover block A or A^{-1} per site), but the
// operands move differently. Every thread copies its own operands of the next hopping
// direction -- its NR = 2 rhs of the 12 neighbour components, 16 bytes each -- into its
// own shared-memory slots with cp.async.cg (L2 -> shared memory, not allocated in L1),
// S - 1 directions ahead of the arithmetic. The first lanes of each site copy the
// direction's link (the 80-byte padded site-major copy) and, with the first direction,
// the site block (site-major copy); the site's lanes read them after a warp barrier
// (the lanes of one site share one warp). Each operand byte is requested from L2 once:
// there are no L1 prefetch hints, whose requests add to those of the loads, and no
// CTA-wide barrier. The self term of pass B is a ninth pipeline item.
#pragma once
#include <mutex>

#include "dslash.cuh"

namespace lqcd {
namespace dpipe {

__device__ __forceinline__ void cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void wait_group() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int kLinkSlot = 10;  // float2 per link in the site-major copy (9 entries + padding)

// Shared memory of one CTA: S stages x 12 components x threads x 16 bytes (spinor slots,
// component-major so that a warp's 16-byte reads are contiguous), S stages x sites x 80
// bytes (links), sites x 288 bytes (site block, when the launch uses one).
template <int S>
__host__ __device__ constexpr size_t smem_bytes(int threads, int sites, bool block) {
  return (size_t)S * 12 * threads * 16 + (size_t)S * sites * kLinkSlot * 8 + (block ? (size_t)sites * 72 * 4 : 0);
}

// One hopping direction (Sec. III-A-1: projection, SU(3) multiply, reconstruction, on (re, im)
// pairs: hop_compute_pairs) from the shared-memory slots of this thread
// (st: component 0 of the stage, stride THREADS float4) and of its site's link (ls: 9 complex
// entries and the padding, read as five 16-byte words), into acc[component][rhs].
template <int MU, int DIR, int THREADS>
__device__ __forceinline__ void hop_smem(const float4* st, const float4* ls, float2 acc[12][2]) {
  float2 u[9];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float4 q = ls[e];
    u[2 * e] = make_float2(q.x, q.y);
    u[2 * e + 1] = make_float2(q.z, q.w);
  }
  u[8] = make_float2(ls[4].x, ls[4].y);
  float2 up[6][2], dn[6][2];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float4 v = st[k * THREADS];
    up[k][0] = make_float2(v.x, v.y);
    up[k][1] = make_float2(v.z, v.w);
    const float4 w = st[(6 + k) * THREADS];
    dn[k][0] = make_float2(w.x, w.y);
    dn[k][1] = make_float2(w.z, w.w);
  }
  hop_compute_pairs<MU, DIR>(u, up, dn, acc);
}

// Quotient of a 32-bit n by d >= 2 from m = ceil(2^64 / d): floor(m n / 2^64) is exact for
// every 32-bit n (Lemire, Kaser and Kurz, "Faster remainder by direct computation", 2019).
__device__ __forceinline__ int fdiv(int n, uint64_t m) { return (int)__umul64hi(m, (uint64_t)(unsigned)n); }
__host__ inline uint64_t fdiv_magic(int d) { return ~uint64_t(0) / (uint64_t)d + 1; }

// site_coords (common.cuh) with the three divisions done by multiply-high.
__device__ __forceinline__ Coord site_coords_fast(const DslashArgs<float>& a, int p, int cb) {
  Coord c;
  const int l2 = cb << 1;
  const int q1 = fdiv(l2, a.div_x);
  const int x0 = l2 - q1 * a.g.X;
  const int q2 = fdiv(q1, a.div_y);
  c.y = q1 - q2 * a.g.Y;
  c.t = fdiv(q2, a.div_z);
  c.z = q2 - c.t * a.g.Z;
  c.x = x0 + ((p + c.t + c.z + c.y) & 1);
  c.lex = l2 - x0 + c.x;
  return c;
}

template <int SELF, int POST, int NRHS, int MAXT, int MINB, int S>
__global__ void __launch_bounds__(MAXT, MINB) dslash_pipe_kernel(DslashArgs<float> a) {
  constexpr int NR = 2;
  constexpr int G = NRHS / NR;  // lanes of one site, all in one warp
  static_assert(32 % G == 0 && S >= 2, "a site's lanes share a warp; at least two stages");
  constexpr int NITEMS = SELF != SELF_NONE ? 9 : 8;
  constexpr bool BLOCK = SELF == SELF_BLOCK || POST == POST_BLOCKINV;
  extern __shared__ __align__(16) unsigned char smem[];
  if (a.skip != nullptr && *a.skip != 0) return;  // the same for every thread of the grid
  // the launch shape is (G, MAXT / G): shared-memory offsets are compile-time constants
  constexpr int threads = MAXT, sites = MAXT / G;
  const int lane = threadIdx.x, tid = threadIdx.y * G + lane;
  float4* sp = reinterpret_cast<float4*>(smem) + tid;
  float2* sl = reinterpret_cast<float2*>(smem + (size_t)S * 12 * threads * 16);
  float* sb = reinterpret_cast<float*>(smem + (size_t)S * 12 * threads * 16 + (size_t)S * sites * kLinkSlot * 8);

  const int site = blockIdx.x * sites + threadIdx.y;
  const bool active = site < a.n_target;
  int p, cb;
  if (a.full) {
    p = (active && site >= a.g.Vh) ? 1 : 0;
    cb = active ? site - p * a.g.Vh : 0;
  } else {
    p = a.target_parity;
    cb = active ? site : 0;
  }
  const int eo_site = p * a.g.Vh + cb;
  const float2* hin = a.hop_in + (a.full ? (1 - p) * a.half_elems : 0);
  const int64_t base = a.full ? p * a.half_elems : 0;

  // neighbour cb index and link site of the eight directions (t+, t-, z+, z-, y+, y-, x+, x-)
  int ncb[8], lsite[8];
  {
    const Coord c = site_coords_fast(a, p, cb);
    const int here = eo_site, there = (1 - p) * a.g.Vh;
    ncb[0] = neighbour_lex<0, +1>(a.g, c) >> 1; lsite[0] = here;
    ncb[1] = neighbour_lex<0, -1>(a.g, c) >> 1; lsite[1] = there + ncb[1];
    ncb[2] = neighbour_lex<1, +1>(a.g, c) >> 1; lsite[2] = here;
    ncb[3] = neighbour_lex<1, -1>(a.g, c) >> 1; lsite[3] = there + ncb[3];
    ncb[4] = neighbour_lex<2, +1>(a.g, c) >> 1; lsite[4] = here;
    ncb[5] = neighbour_lex<2, -1>(a.g, c) >> 1; lsite[5] = there + ncb[5];
    ncb[6] = neighbour_lex<3, +1>(a.g, c) >> 1; lsite[6] = here;
    ncb[7] = neighbour_lex<3, -1>(a.g, c) >> 1; lsite[7] = there + ncb[7];
  }
  const float2* links = static_cast<const float2*>(a.links_aos);

  // copies of pipeline item `item` (directions 0..7, then the self-term input) into stage item % S
  auto issue = [&](int item) {
    if (active && item < NITEMS) {
      float4* st = sp + (item % S) * 12 * threads;
      const float2* src = item < 8 ? hin + (int64_t)ncb[item < 8 ? item : 0] * 12 * NRHS
                                   : a.self_in + base + (int64_t)cb * 12 * NRHS;
      src += lane * NR;
#pragma unroll
      for (int k = 0; k < 12; ++k) cp16(st + k * threads, src + k * NRHS);
      if (item < 8 && lane < kLinkSlot / 2) {
        const int it = item < 8 ? item : 0;
        const float2* lp = links + ((int64_t)(it >> 1) * a.g.V + lsite[it]) * kLinkSlot;
        cp16(sl + ((item % S) * sites + threadIdx.y) * kLinkSlot + 2 * lane, lp + 2 * lane);
      }
    }
    commit();
  };

  // the site block (A for the self term, A^{-1} after the sum) joins the first group
  if (BLOCK && active) {
    const float* blk =
        static_cast<const float*>(POST == POST_BLOCKINV ? a.blocks_inv_aos : a.blocks_aos) + (int64_t)eo_site * 72;
    for (int q = lane; q < 18; q += G) cp16(sb + threadIdx.y * 72 + 4 * q, blk + 4 * q);
  }
#pragma unroll
  for (int s = 0; s < S - 1; ++s) issue(s);

  float2 accp[12][NR];
  MC<float, NR> self[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) accp[k][0] = accp[k][1] = make_float2(0.f, 0.f);

#pragma unroll
  for (int item = 0; item < NITEMS; ++item) {
    __syncwarp();  // the site's lanes are done with the slots the next copies overwrite
    issue(item + S - 1);
    wait_group<S - 1>();
    __syncwarp();  // the link and block copies of the site's first lanes are visible to all its lanes
    if (active) {
      const float4* st = sp + (item % S) * 12 * threads;
      const float4* ls = reinterpret_cast<const float4*>(sl + ((item % S) * sites + threadIdx.y) * kLinkSlot);
      switch (item) {
        case 0: hop_smem<0, +1, threads>(st, ls, accp); break;
        case 1: hop_smem<0, -1, threads>(st, ls, accp); break;
        case 2: hop_smem<1, +1, threads>(st, ls, accp); break;
        case 3: hop_smem<1, -1, threads>(st, ls, accp); break;
        case 4: hop_smem<2, +1, threads>(st, ls, accp); break;
        case 5: hop_smem<2, -1, threads>(st, ls, accp); break;
        case 6: hop_smem<3, +1, threads>(st, ls, accp); break;
        case 7: hop_smem<3, -1, threads>(st, ls, accp); break;
        default:
#pragma unroll
          for (int k = 0; k < 12; ++k) {
            const float4 v = st[k * threads];
            self[k].re[0] = v.x; self[k].im[0] = v.y; self[k].re[1] = v.z; self[k].im[1] = v.w;
          }
      }
    }
  }
  wait_group<0>();
  if (!active) return;

  // scale the hopping sum by c_hop and add the self term: for A psi (pass B) one packed FMA
  // per complex number, c_hop * hop + (A psi)
  MC<float, NR> acc[12];
  const float2 ch = make_float2(a.c_hop, a.c_hop);
  const float* bl = sb + threadIdx.y * 72;
  MC<float, NR> t[12];
  if (SELF == SELF_BLOCK) {
    block_matvec<float, NR>(bl, self, t);
    block_matvec<float, NR>(bl + 36, self + 6, t + 6);
  }
#pragma unroll
  for (int k = 0; k < 12; ++k)
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      float2 v;
      if (SELF == SELF_BLOCK) {
        v = __ffma2_rn(accp[k][q], ch, make_float2(t[k].re[q], t[k].im[q]));
      } else {
        v = __fmul2_rn(accp[k][q], ch);
        if (SELF == SELF_SCALAR) {
          const float2 ss = make_float2(a.self_scalar, a.self_scalar);
          v = __ffma2_rn(ss, make_float2(self[k].re[q], self[k].im[q]), v);
        }
      }
      acc[k].re[q] = v.x;
      acc[k].im[q] = v.y;
    }
  float2* op = a.out + base + (int64_t)cb * 12 * NRHS + lane * NR;
  if (POST == POST_BLOCKINV) {
    block_matvec<float, NR>(bl, acc, t);
    block_matvec<float, NR>(bl + 36, acc + 6, t + 6);
#pragma unroll
    for (int k = 0; k < 12; ++k) mc_store(op + k * NRHS, t[k]);
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      if (POST == POST_SCALAR) {
#pragma unroll
        for (int q = 0; q < NR; ++q) { acc[k].re[q] *= a.post_scalar; acc[k].im[q] *= a.post_scalar; }
      }
      mc_store(op + k * NRHS, acc[k]);
    }
  }
}

template <int SELF, int POST, int NRHS, int MAXT, int MINB, int S>
cudaError_t launch_pipe_one(const DslashArgs<float>& a, cudaStream_t stream) {
  constexpr int G = NRHS / 2;
  const dim3 block(G, MAXT / G);
  const size_t smem = smem_bytes<S>(MAXT, MAXT / G, SELF == SELF_BLOCK || POST == POST_BLOCKINV);
  auto kern = dslash_pipe_kernel<SELF, POST, NRHS, MAXT, MINB, S>;
  static std::once_flag attr;
  std::call_once(attr, [&] {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<S>(MAXT, MAXT / G, true));
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  });
  const dim3 grid((a.n_target + block.y - 1) / block.y);
  DslashArgs<float> b = a;
  b.div_x = fdiv_magic(a.g.X);
  b.div_y = fdiv_magic(a.g.Y);
  b.div_z = fdiv_magic(a.g.Z);
  kern<<<grid, block, smem, stream>>>(b);
  return cudaGetLastError();
}

}  // namespace dpipe

// One pipelined variant: NRHS rhs (16, 32 or 64; a site tile of one site), MAXT threads per
// CTA, at least MINB CTAs per SM, S pipeline stages.
template <int NRHS, int MAXT, int MINB, int S>
cudaError_t launch_dslash_pipe(const DslashArgs<float>& a, int self_mode, int post_mode, cudaStream_t s) {
  if (a.lay.nrhs != NRHS || a.lay.log_s != 0 || a.links_aos == nullptr) return cudaErrorInvalidValue;
  if ((self_mode == SELF_BLOCK && a.blocks_aos == nullptr) ||
      (post_mode == POST_BLOCKINV && a.blocks_inv_aos == nullptr))
    return cudaErrorInvalidValue;
#define LQCD_DP(SMODE, PMODE)                                            \
  if (self_mode == SMODE && post_mode == PMODE)                          \
    return dpipe::launch_pipe_one<SMODE, PMODE, NRHS, MAXT, MINB, S>(a, s);
  LQCD_DP(SELF_SCALAR, POST_NONE)
  LQCD_DP(SELF_BLOCK, POST_NONE)
  LQCD_DP(SELF_NONE, POST_SCALAR)
  LQCD_DP(SELF_NONE, POST_BLOCKINV)
  LQCD_DP(SELF_SCALAR, POST_SCALAR)
  LQCD_DP(SELF_SCALAR, POST_BLOCKINV)
#undef LQCD_DP
  return cudaErrorInvalidValue;
}

#define LQCD_DSLASH_PIPE_TU(NRHS, MAXT, MINB, S) \
  template cudaError_t launch_dslash_pipe<NRHS, MAXT, MINB, S>(const DslashArgs<float>&, int, int, cudaStream_t);

}  // namespace lqcd
