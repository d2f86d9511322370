// Multi-rhs Wilson(-clover) hopping kernel (Sec. III-A-1, Algorithm 1, Eq. (1)-(2)).
//
// One kernel computes, for every target site x and every rhs,
//   out(x) = POST( SELF(self_in)(x) + c_hop * H(hop_in)(x) ),
//   H(psi)(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ],
// SELF in {none, sigma * 1, A(x)}, POST in {none, tau * 1, A(x)^{-1}}. With
// c_hop = -1/2 this is the paper's D = (4 + m0) - C - sum_mu [pi^- U + pi^+ U^dag]
// (pi^+- = (1 +- gamma)/2). The odd-even passes of Sec. III-A-2 are the same
// kernel restricted to one parity:
//   pass A  t_e = A_ee^{-1} D_eo psi_o:  SELF none,  c_hop = -1/2, POST A^{-1}
//   pass B  out = A_oo psi_o - D_oe t_e: SELF A,     c_hop = +1/2, POST none
//   prepare hat b_o = b_o - D_oe u_e:    SELF 1,     c_hop = +1/2
//   reconstruct x_e = A^{-1}(b_e - D_eo x_o): SELF 1, c_hop = +1/2, POST A^{-1}
//
// GPU mapping. Thread (site, rhs group): threadIdx.x picks NR consecutive rhs,
// threadIdx.y the site. The packed spinor layout stores the rhs innermost, so
// the threads of one site read one contiguous run per spin-colour component
// (16-byte vector loads for NR = 2 in FP32 and for FP64), and every lane of a
// site loads the same link and clover entries: the warp broadcasts them, which
// is the paper's "link read once per b rhs". Spin projection (Algorithm 1's
// lambda/chi with 6 of 12 components), the SU(3) multiply on the two projected
// spin components and the reconstruction to 12 components all stay in
// registers; the half spinors are never written to memory. Neighbour halos come
// from L1/L2: each spinor is used by its eight neighbours, which the lexicographic
// thread order keeps within a few time slices, well inside the 129 MB L2.
#pragma once
#include <type_traits>
#include <cuda_bf16.h>

#include <atomic>
#include <mutex>

#include "common.cuh"

namespace lqcd {

enum { SELF_NONE = 0, SELF_SCALAR = 1, SELF_BLOCK = 2 };
enum { POST_NONE = 0, POST_SCALAR = 1, POST_BLOCKINV = 2 };

template <typename Real>
struct DslashArgs {
  using C = typename Cplx<Real>::T;
  Geom g;
  PackedLayout lay;
  int n_target;        // V (full) or V/2 (one parity)
  int full;            // 1: targets are all sites, blocks hold even then odd half
  int target_parity;   // parity of the targets when full == 0
  int hop;             // 0: skip the hopping term (site-local operator only)
  int64_t half_elems;  // complex elements in one parity's half of a packed block
  C* out;
  const C* self_in;    // indexed like out
  const C* hop_in;     // full: full block; else the block of the opposite parity
  const C* links;      // [4][9][V] complex, eo site order, time boundary factor folded in
  const Real* blocks;      // A(x): 72 reals per site, SoA in 16-byte chunks [72*sizeof/16][V]
  const Real* blocks_inv;  // A(x)^{-1}, same layout
  Real self_scalar, post_scalar, c_hop;
  const int* skip;     // optional: return at once when *skip != 0
  int loop_chunk;      // persistent variants: target sites per CTA (set by the launcher)
  int num_sms;         // SMs of the context's device (persistent variants size their grid by it)
  // FP32 copies for the bulk-copy ring kernel (dslash_ring.cuh), null where not built:
  const void* links_aos;       // [4][V][10] float2: each link's 9 entries padded to 80 bytes, eo site order
  const void* blocks_aos;      // [V][72] float: A(x) per site (the 16-byte chunks of `blocks` in site-major order)
  const void* blocks_inv_aos;  // [V][72] float: A(x)^{-1}
  int* err;                    // set (bit 0) when a bounded pipeline wait gives up
  int ring_slots;              // ring kernel: slots per warp (set by its launcher)
  // two-row ("12-real") link copies for FP32 arithmetic, the third row rebuilt in the kernel
  // as conj(row0 x row1) and then multiplied by the time boundary factor where it was folded in:
  const void* links_r12;       // [4][6][V] float2: rows 0, 1 of each packed link
  const void* links_r12_bf16;  // [4][6][V] BF16 pairs: the same rows rounded to BF16
  int link_format;             // 0: 18-real FP32 links (links); 2: 12-real BF16 (links_r12_bf16)
  int blk_rz;                  // > 0: blocked site mapping (ORD = 1 variants, one parity): a CTA takes the
                               // target rows (t, z0 .. z0 + blk_rz - 1, y0 .. y0 + 1); set by the launcher
  Real time_bc;                // fermion time boundary factor (+1 / -1)
  uint64_t div_x, div_y, div_z;  // ceil(2^64 / X), ... : quotients by multiply-high (pipelined kernel; set by its launcher)
};

// NR complex numbers (NR consecutive rhs of one component).
template <typename Real, int NR>
struct MC {
  Real re[NR], im[NR];
};

template <typename Real, int NR>
__device__ __forceinline__ void mc_zero(MC<Real, NR>& a) {
#pragma unroll
  for (int k = 0; k < NR; ++k) { a.re[k] = 0; a.im[k] = 0; }
}

// a += coef * b, coef code: 0 -> +1, 1 -> -1, 2 -> +i, 3 -> -i
template <int CODE, typename Real, int NR>
__device__ __forceinline__ void mc_acc(MC<Real, NR>& a, const MC<Real, NR>& b) {
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    if (CODE == 0) { a.re[k] += b.re[k]; a.im[k] += b.im[k]; }
    if (CODE == 1) { a.re[k] -= b.re[k]; a.im[k] -= b.im[k]; }
    if (CODE == 2) { a.re[k] -= b.im[k]; a.im[k] += b.re[k]; }
    if (CODE == 3) { a.re[k] += b.im[k]; a.im[k] -= b.re[k]; }
  }
}

template <int CODE, typename Real, int NR>
__device__ __forceinline__ MC<Real, NR> mc_comb(const MC<Real, NR>& a, const MC<Real, NR>& b) {
  MC<Real, NR> r = a;
  mc_acc<CODE>(r, b);
  return r;
}

// Vector loads / stores of NR consecutive complex numbers.
__device__ __forceinline__ void mc_load(MC<float, 2>& a, const float2* p) {
  float4 v = __ldg(reinterpret_cast<const float4*>(p));
  a.re[0] = v.x; a.im[0] = v.y; a.re[1] = v.z; a.im[1] = v.w;
}
__device__ __forceinline__ void mc_load(MC<float, 1>& a, const float2* p) {
  float2 v = __ldg(p);
  a.re[0] = v.x; a.im[0] = v.y;
}
__device__ __forceinline__ void mc_load(MC<double, 1>& a, const double2* p) {
  double2 v = __ldg(p);
  a.re[0] = v.x; a.im[0] = v.y;
}
// BF16-stored spinors (pairs re, im), converted to FP32 on load.
__device__ __forceinline__ void mc_load(MC<float, 2>& a, const __nv_bfloat162* p) {
  const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
  __nv_bfloat162 b0, b1;
  memcpy(&b0, &v.x, 4);
  memcpy(&b1, &v.y, 4);
  const float2 c0 = __bfloat1622float2(b0), c1 = __bfloat1622float2(b1);
  a.re[0] = c0.x; a.im[0] = c0.y; a.re[1] = c1.x; a.im[1] = c1.y;
}
__device__ __forceinline__ void mc_load(MC<float, 1>& a, const __nv_bfloat162* p) {
  const float2 c = __bfloat1622float2(__ldg(p));
  a.re[0] = c.x; a.im[0] = c.y;
}

// Loads issued as volatile PTX: they keep their program order, so the link and
// neighbour loads of one direction leave the SM back to back (one memory round
// trip per direction) instead of being spread between the arithmetic.
__device__ __forceinline__ float4 ldg_batch(const float4* p) {
  float4 v;
  asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}
__device__ __forceinline__ float2 ldg_batch(const float2* p) {
  float2 v;
  asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ double2 ldg_batch(const double2* p) {
  double2 v;
  asm volatile("ld.global.nc.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ void mc_load_batch(MC<float, 2>& a, const float2* p) {
  const float4 v = ldg_batch(reinterpret_cast<const float4*>(p));
  a.re[0] = v.x; a.im[0] = v.y; a.re[1] = v.z; a.im[1] = v.w;
}
__device__ __forceinline__ void mc_load_batch(MC<float, 1>& a, const float2* p) {
  const float2 v = ldg_batch(p);
  a.re[0] = v.x; a.im[0] = v.y;
}
__device__ __forceinline__ void mc_load_batch(MC<double, 1>& a, const double2* p) {
  const double2 v = ldg_batch(p);
  a.re[0] = v.x; a.im[0] = v.y;
}

__device__ __forceinline__ void mc_store(float2* p, const MC<float, 2>& a) {
  *reinterpret_cast<float4*>(p) = make_float4(a.re[0], a.im[0], a.re[1], a.im[1]);
}
__device__ __forceinline__ void mc_store(float2* p, const MC<float, 1>& a) {
  *p = make_float2(a.re[0], a.im[0]);
}
__device__ __forceinline__ void mc_store(double2* p, const MC<double, 1>& a) {
  *p = make_double2(a.re[0], a.im[0]);
}

// Spin structure of 1 -+ gamma_mu in the chiral basis gamma = [[0, P], [P^dag, 0]]
// (P_t = 1, P_z = i sigma_z, P_y = i sigma_y, P_x = i sigma_x), with spins
// u0, u1 (upper) and d0, d1 (lower):
//   forward (1 - gamma):  h = u - P d;       lower part of the result = -P^dag (U h)
//   backward (1 + gamma): k = u + P d;       lower part of the result = +P^dag (U^dag k)
// Projection h_s = u_s + coef * d_src, reconstruction low_s += coef * (Uh)_src;
// the backward coefficients are the negatives of the forward ones.
template <int MU> struct SpinTab;
//                       proj: src0 coef0 src1 coef1   recon: src0 coef0 src1 coef1
template <> struct SpinTab<0> { enum { ps0 = 0, pc0 = 1, ps1 = 1, pc1 = 1, rs0 = 0, rc0 = 1, rs1 = 1, rc1 = 1 }; };
template <> struct SpinTab<1> { enum { ps0 = 0, pc0 = 3, ps1 = 1, pc1 = 2, rs0 = 0, rc0 = 2, rs1 = 1, rc1 = 3 }; };
template <> struct SpinTab<2> { enum { ps0 = 1, pc0 = 1, ps1 = 0, pc1 = 0, rs0 = 1, rc0 = 0, rs1 = 0, rc1 = 1 }; };
template <> struct SpinTab<3> { enum { ps0 = 1, pc0 = 3, ps1 = 0, pc1 = 3, rs0 = 1, rc0 = 2, rs1 = 0, rc1 = 2 }; };

__host__ __device__ constexpr int neg_code(int c) { return c == 0 ? 1 : c == 1 ? 0 : c == 2 ? 3 : 2; }

// Complex numbers of one rhs as (re, im) register pairs: the sums of the spin projection and
// of the reconstruction with a coefficient +1 or -1 are packed FP32 adds (add.f32x2; a - b as
// fma.f32x2(b, -1, a), which rounds as the scalar subtraction), the +i / -i ones stay scalar.
// a + coef * b, coef code 0: +1, 1: -1, 2: +i, 3: -i (the codes of SpinTab).
template <int CODE>
__device__ __forceinline__ float2 pcomb(float2 a, float2 b) {
  if constexpr (CODE == 0) return __fadd2_rn(a, b);
  else if constexpr (CODE == 1) return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
  else if constexpr (CODE == 2) return make_float2(a.x - b.y, a.y + b.x);
  else return make_float2(a.x + b.y, a.y - b.x);
}

// The direction of hop_compute below for FP32 and two rhs per thread, on (re, im) pairs: the
// same operations in the same order, the +-1 sums packed.
template <int MU, int DIR>
__device__ __forceinline__ void hop_compute_pairs(const float2* u, const float2 (*up)[2], const float2 (*dn)[2],
                                                  float2 (*acc)[2]) {
  using Tab = SpinTab<MU>;
  constexpr int pc0 = DIR > 0 ? Tab::pc0 : neg_code(Tab::pc0);
  constexpr int pc1 = DIR > 0 ? Tab::pc1 : neg_code(Tab::pc1);
  constexpr int rc0 = DIR > 0 ? Tab::rc0 : neg_code(Tab::rc0);
  constexpr int rc1 = DIR > 0 ? Tab::rc1 : neg_code(Tab::rc1);
  float2 h[6][2];  // [spin s][colour] of the half spinor, per rhs
#pragma unroll
  for (int col = 0; col < 3; ++col)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      h[col][r] = pcomb<pc0>(up[col][r], dn[3 * Tab::ps0 + col][r]);
      h[3 + col][r] = pcomb<pc1>(up[3 + col][r], dn[3 * Tab::ps1 + col][r]);
    }
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int ar = 0; ar < 3; ++ar)
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        float2 o = make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          // forward: U[ar][b] * h_b ; backward: conj(U[b][ar]) * h_b
          const float2 m = (DIR > 0) ? u[3 * ar + b] : u[3 * b + ar];
          const float mr = m.x, mi = (DIR > 0) ? m.y : -m.y;
          const float2 v = h[3 * s + b][r];
          o.x = fmaf(mr, v.x, o.x);
          o.x = fmaf(-mi, v.y, o.x);
          o.y = fmaf(mr, v.y, o.y);
          o.y = fmaf(mi, v.x, o.y);
        }
        acc[3 * s + ar][r] = __fadd2_rn(acc[3 * s + ar][r], o);
        // lower spin 0 takes product spin rs0, lower spin 1 product spin rs1 (a permutation)
        if (Tab::rs0 == s) acc[6 + ar][r] = pcomb<rc0>(acc[6 + ar][r], o);
        else acc[9 + ar][r] = pcomb<rc1>(acc[9 + ar][r], o);
      }
}

// Spin projection, SU(3) multiply and reconstruction of one hopping direction
// (forward for DIR = +1, backward for DIR = -1) from the neighbour spinor (upper
// spins up[6], lower spins dn[6]) and the link u[9] (row-major).
template <typename Real, int NR, int MU, int DIR>
__device__ __forceinline__ void hop_compute(const typename Cplx<Real>::T* u, const MC<Real, NR>* up,
                                            const MC<Real, NR>* dn, MC<Real, NR> acc[12]) {
  if constexpr (std::is_same<Real, float>::value && NR == 2) {
    float2 upp[6][2], dnp[6][2], accp[12][2];
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        upp[k][r] = make_float2(up[k].re[r], up[k].im[r]);
        dnp[k][r] = make_float2(dn[k].re[r], dn[k].im[r]);
      }
#pragma unroll
    for (int k = 0; k < 12; ++k)
#pragma unroll
      for (int r = 0; r < 2; ++r) accp[k][r] = make_float2(acc[k].re[r], acc[k].im[r]);
    hop_compute_pairs<MU, DIR>(u, upp, dnp, accp);
#pragma unroll
    for (int k = 0; k < 12; ++k)
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        acc[k].re[r] = accp[k][r].x;
        acc[k].im[r] = accp[k][r].y;
      }
    return;
  }
  using C = typename Cplx<Real>::T;
  using Tab = SpinTab<MU>;
  constexpr int pc0 = DIR > 0 ? Tab::pc0 : neg_code(Tab::pc0);
  constexpr int pc1 = DIR > 0 ? Tab::pc1 : neg_code(Tab::pc1);
  constexpr int rc0 = DIR > 0 ? Tab::rc0 : neg_code(Tab::rc0);
  constexpr int rc1 = DIR > 0 ? Tab::rc1 : neg_code(Tab::rc1);
  MC<Real, NR> h[6];  // [spin s in 0,1][colour]
#pragma unroll
  for (int col = 0; col < 3; ++col) {
    h[col] = mc_comb<pc0>(up[col], dn[3 * Tab::ps0 + col]);
    h[3 + col] = mc_comb<pc1>(up[3 + col], dn[3 * Tab::ps1 + col]);
  }
  MC<Real, NR> w[6];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
#pragma unroll
    for (int ar = 0; ar < 3; ++ar) {
      MC<Real, NR>& o = w[3 * s + ar];
      mc_zero(o);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        // forward: U[ar][b] * h_b ; backward: conj(U[b][ar]) * h_b
        const C m = (DIR > 0) ? u[3 * ar + b] : u[3 * b + ar];
        const Real mr = m.x;
        const Real mi = (DIR > 0) ? m.y : -m.y;
        const MC<Real, NR>& v = h[3 * s + b];
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          o.re[k] = fma(mr, v.re[k], o.re[k]);
          o.re[k] = fma(-mi, v.im[k], o.re[k]);
          o.im[k] = fma(mr, v.im[k], o.im[k]);
          o.im[k] = fma(mi, v.re[k], o.im[k]);
        }
      }
    }
  }
#pragma unroll
  for (int col = 0; col < 3; ++col) {
    mc_acc<0>(acc[col], w[col]);
    mc_acc<0>(acc[3 + col], w[3 + col]);
    mc_acc<rc0>(acc[6 + col], w[3 * Tab::rs0 + col]);
    mc_acc<rc1>(acc[9 + col], w[3 * Tab::rs1 + col]);
  }
}

// Packed index with the rhs count fixed at compile time (NRHS > 0: a site tile of one
// site, S = 1, which holds for nrhs >= 16): the component offsets become immediates.
template <int NRHS>
__device__ __forceinline__ int64_t lidx(const PackedLayout& lay, int64_t i, int c, int r) {
  if constexpr (NRHS > 0) return (i * 12 + c) * NRHS + r;
  else return lay.index(i, c, r);
}

// Link storage formats of the FP32 kernels: LF = 0 the 18-real links; LF = 1 rows 0 and 1
// in FP32; LF = 2 rows 0 and 1 in BF16. For LF > 0 the third row of the SU(3) matrix is
// rebuilt as conj(row0 x row1); the stored rows carry the time boundary factor b of
// U_0 on the last time slice, which cancels in the cross product (b^2 = 1), so the
// rebuilt row is multiplied by b for those links.
__device__ __forceinline__ float2 cmul_f(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ void rebuild_third_row(float2 u[9], float b) {
  const float2 a0 = cmul_f(u[1], u[5]), a1 = cmul_f(u[2], u[4]);
  const float2 b0 = cmul_f(u[2], u[3]), b1 = cmul_f(u[0], u[5]);
  const float2 c0 = cmul_f(u[0], u[4]), c1 = cmul_f(u[1], u[3]);
  u[6] = make_float2(b * (a0.x - a1.x), -b * (a0.y - a1.y));
  u[7] = make_float2(b * (b0.x - b1.x), -b * (b0.y - b1.y));
  u[8] = make_float2(b * (c0.x - c1.x), -b * (c0.y - c1.y));
}
template <int LF>
__device__ __forceinline__ void load_link_r12(const DslashArgs<float>& a, int mu, int link_site, float2 u[9]) {
  if constexpr (LF == 1) {
    const float2* lp = static_cast<const float2*>(a.links_r12) + (int64_t)(mu * 6) * a.g.V + link_site;
#pragma unroll
    for (int e = 0; e < 6; ++e) u[e] = __ldg(lp + (int64_t)e * a.g.V);
  } else {
    const __nv_bfloat162* lp =
        static_cast<const __nv_bfloat162*>(a.links_r12_bf16) + (int64_t)(mu * 6) * a.g.V + link_site;
#pragma unroll
    for (int e = 0; e < 6; ++e) u[e] = __bfloat1622float2(__ldg(lp + (int64_t)e * a.g.V));
  }
}

// One hopping direction with direct (register) loads of the link and the neighbour
// (BATCH: as one batch of volatile loads).
template <typename Real, int NR, int MU, int DIR, bool BATCH, typename HIN, int NRHS = 0, int LF = 0>
__device__ __forceinline__ void hop_dir(const DslashArgs<Real>& a, const Coord& c, int p, int r0,
                                        const HIN* hin, MC<Real, NR> acc[12]) {
  using C = typename Cplx<Real>::T;
  const int nlex = neighbour_lex<MU, DIR>(a.g, c);
  const int ncb = nlex >> 1;
  // link: U_mu(x) forward, U_mu(x - mu) backward (eo index of its base site)
  const int link_site = (DIR > 0) ? (p * a.g.Vh + (c.lex >> 1)) : ((1 - p) * a.g.Vh + ncb);
  const C* lp = a.links + (int64_t)(MU * 9) * a.g.V + link_site;
  C u[9];
  MC<Real, NR> up[6], dn[6];
  if constexpr (LF > 0) {
    static_assert(sizeof(Real) == 4, "two-row links: FP32 kernels only");
    load_link_r12<LF>(a, MU, link_site, u);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      mc_load(up[k], hin + lidx<NRHS>(a.lay, ncb, k, r0));
      mc_load(dn[k], hin + lidx<NRHS>(a.lay, ncb, 6 + k, r0));
    }
    // the time links of the last time slice carry the boundary factor
    const bool edge = MU == 0 && (DIR > 0 ? c.t == a.g.T - 1 : c.t == 0);
    rebuild_third_row(u, edge ? a.time_bc : 1.f);
  } else if constexpr (BATCH) {
#pragma unroll
    for (int e = 0; e < 9; ++e) u[e] = ldg_batch(lp + (int64_t)e * a.g.V);
#pragma unroll
    for (int k = 0; k < 6; ++k) mc_load_batch(up[k], hin + lidx<NRHS>(a.lay, ncb, k, r0));
#pragma unroll
    for (int k = 0; k < 6; ++k) mc_load_batch(dn[k], hin + lidx<NRHS>(a.lay, ncb, 6 + k, r0));
  } else {
#pragma unroll
    for (int e = 0; e < 9; ++e) u[e] = __ldg(lp + (int64_t)e * a.g.V);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      mc_load(up[k], hin + lidx<NRHS>(a.lay, ncb, k, r0));
      mc_load(dn[k], hin + lidx<NRHS>(a.lay, ncb, 6 + k, r0));
    }
  }
  hop_compute<Real, NR, MU, DIR>(u, up, dn, acc);
}

// L1 prefetch of one hopping direction's operands (the neighbour spinor of this
// site and its link), issued PF directions ahead of their loads in the variants
// compiled for a fixed rhs count (site tile of one site, so a site's spinor is one
// contiguous run of 12 * NRHS complex numbers). The site's NRHS / NR lanes split
// the run's 128-byte lines between them. A prefetch holds no register, so the
// bytes in flight per warp are no longer bounded by the registers that receive
// them; the later loads of that direction then hit L1.
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

template <typename Real, int NR, int MU, int DIR, typename HIN, int NRHS>
__device__ __forceinline__ void prefetch_dir(const DslashArgs<Real>& a, const Coord& c, int p, const HIN* hin) {
  static_assert(NRHS >= 16, "prefetch variants need a site tile of one site");
  constexpr int G = NRHS / NR;                                  // lanes of one site
  constexpr int LINES = 12 * NRHS * (int)sizeof(HIN) / 128;     // lines of one site's spinor
  const int ncb = neighbour_lex<MU, DIR>(a.g, c) >> 1;
  const char* sp = reinterpret_cast<const char*>(hin + (int64_t)ncb * 12 * NRHS);
#pragma unroll
  for (int l = 0; l < (LINES + G - 1) / G; ++l) {
    const int line = (int)threadIdx.x + l * G;
    if (line < LINES) prefetch_l1(sp + line * 128);
  }
  const int link_site = (DIR > 0) ? (p * a.g.Vh + (c.lex >> 1)) : ((1 - p) * a.g.Vh + ncb);
  const typename Cplx<Real>::T* lp = a.links + (int64_t)(MU * 9) * a.g.V + link_site;
#pragma unroll
  for (int l = 0; l < (9 + G - 1) / G; ++l) {
    const int e = (int)threadIdx.x + l * G;
    if (e < 9) prefetch_l1(lp + (int64_t)e * a.g.V);
  }
}

// Direction K = 0..7 of the hopping sum, forward for even K: mu = K / 2 in order t, z, y, x
// (ORD = 0) or mu = 3 - K / 2 in order x, y, z, t (ORD = 1: the directions whose neighbour
// spinors the CTA's other rows share come first, while they are still in L1).
template <int K, int ORD = 0> struct DirOf {
  static constexpr int MU = ORD == 0 ? K / 2 : 3 - K / 2;
  static constexpr int DIR = (K % 2 == 0) ? +1 : -1;
};

template <typename Real, int NR, bool BATCH, typename HIN, int NRHS, int PF, int K, int LF = 0, int ORD = 0>
__device__ __forceinline__ void hop_step(const DslashArgs<Real>& a, const Coord& c, int p, int r0, const HIN* hin,
                                         MC<Real, NR> acc[12]) {
  if constexpr (PF > 0 && K + PF < 8)
    prefetch_dir<Real, NR, DirOf<K + PF, ORD>::MU, DirOf<K + PF, ORD>::DIR, HIN, NRHS>(a, c, p, hin);
  hop_dir<Real, NR, DirOf<K, ORD>::MU, DirOf<K, ORD>::DIR, BATCH, HIN, NRHS, LF>(a, c, p, r0, hin, acc);
}

// Packed Hermitian 6x6 block: 6 real diagonal entries, then the 15 strictly
// lower entries L(l, j), l > j, in the order (1,0), (2,0), (2,1), (3,0), ...
// (index l(l-1)/2 + j) as (re, im) pairs: 36 reals. Site blocks hold the upper
// chiral block (spins 0, 1) then the lower one (spins 2, 3): 72 reals.
template <typename Real, int NR>
__device__ __forceinline__ void block_matvec(const Real* m, const MC<Real, NR>* x, MC<Real, NR>* y) {
#pragma unroll
  for (int l = 0; l < 6; ++l) {
#pragma unroll
    for (int k = 0; k < NR; ++k) { y[l].re[k] = m[l] * x[l].re[k]; y[l].im[k] = m[l] * x[l].im[k]; }
  }
#pragma unroll
  for (int l = 1; l < 6; ++l) {
#pragma unroll
    for (int j = 0; j < l; ++j) {
      const Real lr = m[6 + 2 * (l * (l - 1) / 2 + j)];
      const Real li = m[6 + 2 * (l * (l - 1) / 2 + j) + 1];
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        // y_l += L_lj x_j
        y[l].re[k] = fma(lr, x[j].re[k], y[l].re[k]);
        y[l].re[k] = fma(-li, x[j].im[k], y[l].re[k]);
        y[l].im[k] = fma(lr, x[j].im[k], y[l].im[k]);
        y[l].im[k] = fma(li, x[j].re[k], y[l].im[k]);
        // y_j += conj(L_lj) x_l
        y[j].re[k] = fma(lr, x[l].re[k], y[j].re[k]);
        y[j].re[k] = fma(li, x[l].im[k], y[j].re[k]);
        y[j].im[k] = fma(lr, x[l].im[k], y[j].im[k]);
        y[j].im[k] = fma(-li, x[l].re[k], y[j].im[k]);
      }
    }
  }
}

// Load one chiral half (36 reals) of a site's packed block.
__device__ __forceinline__ void load_half_block(float* dst, const float* blocks, int V, int site, int half) {
  const float4* b4 = reinterpret_cast<const float4*>(blocks);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    float4 v = __ldg(b4 + (int64_t)(9 * half + k) * V + site);
    dst[4 * k] = v.x; dst[4 * k + 1] = v.y; dst[4 * k + 2] = v.z; dst[4 * k + 3] = v.w;
  }
}
__device__ __forceinline__ void load_half_block(double* dst, const double* blocks, int V, int site, int half) {
  const double2* b2 = reinterpret_cast<const double2*>(blocks);
#pragma unroll
  for (int k = 0; k < 18; ++k) {
    double2 v = __ldg(b2 + (int64_t)(18 * half + k) * V + site);
    dst[2 * k] = v.x; dst[2 * k + 1] = v.y;
  }
}

template <typename Real, int NR>
__device__ __forceinline__ void site_block_apply(const Real* blocks, int V, int site,
                                                 const MC<Real, NR> x[12], MC<Real, NR> y[12]) {
  Real m[36];
  load_half_block(m, blocks, V, site, 0);
  block_matvec<Real, NR>(m, x, y);
  load_half_block(m, blocks, V, site, 1);
  block_matvec<Real, NR>(m, x + 6, y + 6);
}

// The whole operator on one target site for this thread's NR rhs.
template <typename Real, int NR, int SELF, int POST, bool BATCH, typename HIN, typename SIN, int NRHS = 0, int PF = 0,
          int LF = 0, int ORD = 0>
__device__ __forceinline__ void dslash_site(const DslashArgs<Real>& a, int site) {
  using C = typename Cplx<Real>::T;
  const int r0 = threadIdx.x * NR;
  int p, cb;
  if (a.full) {
    p = site >= a.g.Vh ? 1 : 0;
    cb = site - p * a.g.Vh;
  } else {
    p = a.target_parity;
    cb = site;
  }
  const int eo_site = p * a.g.Vh + cb;

  MC<Real, NR> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) mc_zero(acc[k]);

  if (a.hop) {
    const Coord c = site_coords(a.g, p, cb);
    const HIN* hin = reinterpret_cast<const HIN*>(a.hop_in) + (a.full ? (1 - p) * a.half_elems : 0);
    if constexpr (PF > 0) {
      prefetch_dir<Real, NR, DirOf<0, ORD>::MU, +1, HIN, NRHS>(a, c, p, hin);
      if constexpr (PF > 1) prefetch_dir<Real, NR, DirOf<1, ORD>::MU, -1, HIN, NRHS>(a, c, p, hin);
    }
    hop_step<Real, NR, BATCH, HIN, NRHS, PF, 0, LF, ORD>(a, c, p, r0, hin, acc);
    hop_step<Real, NR, BATCH, HIN, NRHS, PF, 1, LF, ORD>(a, c, p, r0, hin, acc);
    hop_step<Real, NR, BATCH, HIN, NRHS, PF, 2, LF, ORD>(a, c, p, r0, hin, acc);
    hop_step<Real, NR, BATCH, HIN, NRHS, PF, 3, LF, ORD>(a, c, p, r0, hin, acc);
    hop_step<Real, NR, BATCH, HIN, NRHS, PF, 4, LF, ORD>(a, c, p, r0, hin, acc);
    hop_step<Real, NR, BATCH, HIN, NRHS, PF, 5, LF, ORD>(a, c, p, r0, hin, acc);
    hop_step<Real, NR, BATCH, HIN, NRHS, PF, 6, LF, ORD>(a, c, p, r0, hin, acc);
    hop_step<Real, NR, BATCH, HIN, NRHS, PF, 7, LF, ORD>(a, c, p, r0, hin, acc);
#pragma unroll
    for (int k = 0; k < 12; ++k)
#pragma unroll
      for (int q = 0; q < NR; ++q) { acc[k].re[q] *= a.c_hop; acc[k].im[q] *= a.c_hop; }
  }

  const int64_t base = a.full ? p * a.half_elems : 0;
  if (SELF != SELF_NONE) {
    const SIN* sp = reinterpret_cast<const SIN*>(a.self_in) + base;
    MC<Real, NR> s[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) mc_load(s[k], sp + lidx<NRHS>(a.lay, cb, k, r0));
    if (SELF == SELF_SCALAR) {
#pragma unroll
      for (int k = 0; k < 12; ++k)
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          acc[k].re[q] = fma(a.self_scalar, s[k].re[q], acc[k].re[q]);
          acc[k].im[q] = fma(a.self_scalar, s[k].im[q], acc[k].im[q]);
        }
    } else {
      MC<Real, NR> t[12];
      site_block_apply<Real, NR>(a.blocks, a.g.V, eo_site, s, t);
#pragma unroll
      for (int k = 0; k < 12; ++k)
#pragma unroll
        for (int q = 0; q < NR; ++q) { acc[k].re[q] += t[k].re[q]; acc[k].im[q] += t[k].im[q]; }
    }
  }

  C* op = a.out + base;
  if (POST == POST_BLOCKINV) {
    MC<Real, NR> t[12];
    site_block_apply<Real, NR>(a.blocks_inv, a.g.V, eo_site, acc, t);
#pragma unroll
    for (int k = 0; k < 12; ++k) mc_store(op + lidx<NRHS>(a.lay, cb, k, r0), t[k]);
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      if (POST == POST_SCALAR) {
#pragma unroll
        for (int q = 0; q < NR; ++q) { acc[k].re[q] *= a.post_scalar; acc[k].im[q] *= a.post_scalar; }
      }
      mc_store(op + lidx<NRHS>(a.lay, cb, k, r0), acc[k]);
    }
  }
}

template <typename Real, int NR, int SELF, int POST, int MAXT, int MINB, bool BATCH, bool LOOP, typename HIN,
          typename SIN, int NRHS = 0, int PF = 0, int LF = 0, int ORD = 0>
__global__ void __launch_bounds__(MAXT, MINB) dslash_kernel(DslashArgs<Real> a) {
  if (a.skip != nullptr && *a.skip != 0) return;
  if (!LOOP) {
    int site = blockIdx.x * blockDim.y + threadIdx.y;
    if (ORD == 1 && a.blk_rz > 0) {
      // blocked mapping (one parity): the CTA's targets are the X/2 targets of each of the rows
      // (t, z0 + dz, y0 + dy), dz < blk_rz, dy < 2, so the rows' shared neighbour spinors meet in L1
      const int hx = a.g.X >> 1;
      const int xi = threadIdx.y % hx, row = threadIdx.y / hx;
      const int ny = a.g.Y >> 1, nz = a.g.Z / a.blk_rz;
      int b = blockIdx.x;
      const int yb = b % ny;
      b /= ny;
      const int zb = b % nz, t = b / nz;
      const int z = zb * a.blk_rz + (row >> 1), y = yb * 2 + (row & 1);
      site = ((((t * a.g.Z + z) * a.g.Y + y) * a.g.X) >> 1) + xi;
    }
    if (site < a.n_target) dslash_site<Real, NR, SELF, POST, BATCH, HIN, SIN, NRHS, PF, LF, ORD>(a, site);
    return;
  }
  // persistent CTAs: each walks one contiguous chunk of target sites, blockDim.y
  // sites at a time, so the neighbour rows in x and y it loaded for the previous
  // sites are still in L1 for the next ones
  const int s0 = blockIdx.x * a.loop_chunk;
  const int s1 = min(s0 + a.loop_chunk, a.n_target);
  for (int site = s0 + threadIdx.y; site < s1; site += blockDim.y)
    dslash_site<Real, NR, SELF, POST, BATCH, HIN, SIN, NRHS, PF, LF, ORD>(a, site);
}

// Launch variants of the kernel: rhs per thread (NR), threads per CTA (the CTA is
// nrhs/NR threads wide and threads/(nrhs/NR) sites tall) and a minimum number of
// resident CTAs per SM (which caps the registers per thread). The autotuner
// (lqcd_tune) times them; variant -1 is the built-in default.
struct DslashVariant {
  int nr, threads, minb;
  int stages;  // 0: direct register loads; >= 2: cp.async pipeline depth (dslash_async.cuh)
  int batch;   // direct loads: 1 = each direction's loads issued as one batch
  int loop;    // direct loads: 1 = persistent CTAs walking contiguous chunks of sites
  int nrhs_fixed = 0;  // > 0: compiled for this rhs count only (immediate component offsets)
  int prefetch = 0;    // with nrhs_fixed: L1 prefetch of the operands this many directions ahead
  int ring_warps = 0;  // > 0: the bulk-copy ring kernel (dslash_ring.cuh) with this many warps per CTA
  int ring_slots = 0;  //       and this many ring slots per warp
  int links = 0;       // 1: reads the 12-real FP32 link copy (third row rebuilt)
  int order = 0;       // 1: directions x, y, z, t and the blocked site mapping (one CTA per row block)
  int pipe = 0;        // > 0: the pipelined kernel (dslash_pipe.cuh) with this many cp.async stages
};
int dslash_variant_count(bool f64);
DslashVariant dslash_variant(bool f64, int idx);
int dslash_default_variant(bool f64, int nrhs);
bool dslash_variant_ok(bool f64, int idx, int nrhs);

template <typename Real>
cudaError_t launch_dslash(const DslashArgs<Real>& a, int self_mode, int post_mode, int variant,
                          cudaStream_t stream);

// Launch one (SELF, POST) combination of one variant; defined by LQCD_DSLASH_VARIANT_TU.
template <typename Real, int NR, int SM, int PM, int MAXT, int MINB, bool BATCH, bool LOOP, typename HIN,
          typename SIN, int NRHS = 0, int PF = 0, int LF = 0, int ORD = 0>
cudaError_t launch_dslash_one(DslashArgs<Real> a, dim3 block, cudaStream_t s) {
  auto kern = dslash_kernel<Real, NR, SM, PM, MAXT, MINB, BATCH, LOOP, HIN, SIN, NRHS, PF, LF, ORD>;
  dim3 grid((a.n_target + block.y - 1) / block.y);
  a.blk_rz = 0;
  if (ORD == 1 && !LOOP && !a.full) {
    // the blocked mapping needs whole rows per CTA, an even row count and z blocks that tile Z
    const int hx = a.g.X / 2;
    const int rows = hx > 0 && (int)block.y % hx == 0 ? (int)block.y / hx : 0;
    if (rows >= 2 && rows % 2 == 0 && a.g.X % 2 == 0 && a.g.Y % 2 == 0 && a.g.Z % (rows / 2) == 0 &&
        a.n_target == a.g.Vh && (int)grid.x * (int)block.y == a.n_target)
      a.blk_rz = rows / 2;
  }
  if (PF > 0) {
    // the prefetched lines live in L1: ask for the smallest shared-memory carve-out
    static std::once_flag carveout;
    std::call_once(carveout, [&] { cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 0); });
  }
  if (LOOP) {
    // one wave of persistent CTAs, each with an equal contiguous chunk of sites; the
    // resident-CTA count depends only on the kernel and the architecture, the SM count
    // comes from the context's device
    static std::atomic<int> per_sm_cache{0};
    int per_sm = per_sm_cache.load(std::memory_order_relaxed);
    if (per_sm == 0) {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block.x * block.y, 0);
      if (per_sm < 1) per_sm = 1;
      per_sm_cache.store(per_sm, std::memory_order_relaxed);
    }
    const int want = (a.num_sms > 0 ? a.num_sms : 1) * per_sm;
    const int rows = (int)grid.x;
    const int per_cta = (rows + want - 1) / want;
    a.loop_chunk = per_cta * (int)block.y;
    grid.x = (a.n_target + a.loop_chunk - 1) / a.loop_chunk;
  }
  kern<<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename Real, int NR, int MAXT, int MINB, bool BATCH, bool LOOP = false,
          typename HIN = typename Cplx<Real>::T, typename SIN = typename Cplx<Real>::T, int NRHS = 0, int PF = 0,
          int LF = 0, int ORD = 0>
cudaError_t launch_dslash_variant(const DslashArgs<Real>& a, int self_mode, int post_mode, cudaStream_t s) {
  if (NRHS > 0 && (a.lay.nrhs != NRHS || a.lay.log_s != 0)) return cudaErrorInvalidValue;
  if (LF == 1 && a.links_r12 == nullptr) return cudaErrorInvalidValue;
  if (LF == 2 && a.links_r12_bf16 == nullptr) return cudaErrorInvalidValue;
  const int G = a.lay.nrhs / NR;
  dim3 block(G, G >= MAXT ? 1 : MAXT / G);
#define LQCD_DS(SM, PM) \
  return launch_dslash_one<Real, NR, SM, PM, MAXT, MINB, BATCH, LOOP, HIN, SIN, NRHS, PF, LF, ORD>(a, block, s)
  if (self_mode == SELF_SCALAR && post_mode == POST_NONE) LQCD_DS(SELF_SCALAR, POST_NONE);
  else if (self_mode == SELF_BLOCK && post_mode == POST_NONE) LQCD_DS(SELF_BLOCK, POST_NONE);
  else if (self_mode == SELF_NONE && post_mode == POST_SCALAR) LQCD_DS(SELF_NONE, POST_SCALAR);
  else if (self_mode == SELF_NONE && post_mode == POST_BLOCKINV) LQCD_DS(SELF_NONE, POST_BLOCKINV);
  else if (self_mode == SELF_SCALAR && post_mode == POST_SCALAR) LQCD_DS(SELF_SCALAR, POST_SCALAR);
  else if (self_mode == SELF_SCALAR && post_mode == POST_BLOCKINV) LQCD_DS(SELF_SCALAR, POST_BLOCKINV);
  else return cudaErrorInvalidValue;
#undef LQCD_DS
}

// Explicit instantiation of one variant's launcher in its own translation unit
// (the variants compile in parallel).
#define LQCD_DSLASH_VARIANT_TU(REAL, NR, MAXT, MINB, BATCH, LOOP) \
  template cudaError_t launch_dslash_variant<REAL, NR, MAXT, MINB, BATCH, LOOP>(const DslashArgs<REAL>&, int, int, cudaStream_t);
// ... and of a variant with the rhs count fixed at compile time.
#define LQCD_DSLASH_VARIANT_NRHS_TU(REAL, NR, MAXT, MINB, NRHS, PF)                                        \
  template cudaError_t launch_dslash_variant<REAL, NR, MAXT, MINB, false, false, typename Cplx<REAL>::T, \
                                             typename Cplx<REAL>::T, NRHS, PF>(const DslashArgs<REAL>&, int, int, cudaStream_t);

// ... and of an FP32 variant reading two-row links (LF = 1: FP32 rows, 2: BF16 rows).
#define LQCD_DSLASH_VARIANT_LF_TU(NR, MAXT, MINB, LOOP, NRHS, PF, LF)                                      \
  template cudaError_t launch_dslash_variant<float, NR, MAXT, MINB, false, LOOP, float2, float2, NRHS, PF, LF>( \
      const DslashArgs<float>&, int, int, cudaStream_t);

// ... and of an FP32 variant with the blocked mapping and the x, y, z, t direction order.
#define LQCD_DSLASH_VARIANT_ORD_TU(NR, MAXT, MINB, NRHS, PF)                                                  \
  template cudaError_t launch_dslash_variant<float, NR, MAXT, MINB, false, false, float2, float2, NRHS, PF, 0, 1>( \
      const DslashArgs<float>&, int, int, cudaStream_t);

// FP32 arithmetic on BF16-stored inputs (hop input HIN, self-term input SIN), FP32 output.
cudaError_t launch_dslash_bf16(const DslashArgs<float>& a, int self_mode, int post_mode, bool hop_bf16,
                               cudaStream_t stream);

}  // namespace lqcd
