// Batched restarted GMRES (Algorithm 2) on the GPU, with optional odd-even
// preconditioning (Sec. III-A-2) and FP32-inside-FP64 iterative refinement.
//
// Structure of one solve (every rhs independent, as in the paper's batched solver):
//   restart: r = b - D x in FP64 (FP64 operator), ||r|| per rhs; the host reads
//            the norms (one stream synchronisation per restart), retires the rhs
//            whose true residual meets tol, and starts a cycle for the others
//            with v_0 = r / ||r|| stored in the inner precision;
//   cycle:   m Arnoldi steps, each = operator apply (inner precision) + block
//            classical Gram-Schmidt with one re-orthogonalisation (CGS2, fused
//            dot/update passes) + a device kernel that updates the Hessenberg
//            column with the stored Givens rotations, forms the new rotation and
//            gamma, and tests |gamma_{j+1}| against the cycle threshold per rhs
//            (rhs that met it stop contributing: their next basis vector is 0);
//            the whole cycle can be replayed as one captured CUDA graph;
//   update:  back substitution (FP64, device) and x += V y with x in FP64.
// In FP64 mode the inner precision is FP64 and this is plain restarted GMRES;
// in FP32 mode it is GMRES-based iterative refinement: FP64 stays on the true
// residual, the solution update and the small Givens / least-squares step.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"

namespace lqcd {

// ------------------------------------------------------------------ small dense kernels

__global__ void cycle_init_kernel(GmresState s, const double* __restrict__ beta0) {
  const int r = threadIdx.x;
  bool live = false;
  if (r < s.nrhs) {
    const int act = s.active[r];
    for (int i = 0; i <= s.m; ++i) s.gamma[(int64_t)r * (s.m + 1) + i] = make_double2(0, 0);
    s.gamma[(int64_t)r * (s.m + 1)] = make_double2(act ? beta0[r] : 0.0, 0.0);
    s.done[r] = act ? 0 : 1;
    s.k[r] = 0;
    s.scale[r] = act ? 1.0 / beta0[r] : 0.0;
    live = act != 0;
  }
  const int any = __syncthreads_or(live);
  if (threadIdx.x == 0) {
    *s.all_done = any ? 0 : 1;
    *s.kmax = 0;
  }
}

// Givens step for Hessenberg column j of rhs r: the stored rotations applied to
// col[0..j], a new rotation (c = |a|/rho, s = (a/|a|) beta/rho) against the
// sub-diagonal entry beta, gamma_{j+1} = -conj(s) gamma_j, gamma_j = c gamma_j,
// and the stop test (|gamma_{j+1}| <= thr, happy breakdown beta <= 1e-14 ||column||,
// the last column, or a non-finite value). Returns whether the cycle goes on.
// cs_prev / sn_prev: optional copies of the earlier rotations (e.g. staged in shared memory).
__device__ bool givens_step(const GmresState& s, int r, int j, double2* col, double beta, double w2,
                            const double* cs_prev = nullptr, const double2* sn_prev = nullptr) {
  double* cs = s.cs + (int64_t)r * s.m;
  double2* sn = s.sn + (int64_t)r * s.m;
  const double* csr = cs_prev ? cs_prev : cs;
  const double2* snr = sn_prev ? sn_prev : sn;
  for (int i = 0; i < j; ++i) {
    const double2 top = col[i], bot = col[i + 1];
    const double c = csr[i];
    const double2 sv = snr[i];
    // top' = c top + s bot ; bot' = -conj(s) top + c bot
    col[i] = make_double2(c * top.x + sv.x * bot.x - sv.y * bot.y, c * top.y + sv.x * bot.y + sv.y * bot.x);
    col[i + 1] = make_double2(-(sv.x * top.x + sv.y * top.y) + c * bot.x,
                              -(sv.x * top.y - sv.y * top.x) + c * bot.y);
  }
  const double2 a = col[j];
  const double aa = hypot(a.x, a.y);
  const double rho = hypot(aa, beta);
  double c;
  double2 sv, rjj;
  if (rho == 0.0) {
    c = 1.0; sv = make_double2(0, 0); rjj = make_double2(0, 0);
  } else if (aa == 0.0) {
    c = 0.0; sv = make_double2(1, 0); rjj = make_double2(rho, 0);
  } else {
    const double2 ph = make_double2(a.x / aa, a.y / aa);
    c = aa / rho;
    sv = make_double2(ph.x * beta / rho, ph.y * beta / rho);
    rjj = make_double2(ph.x * rho, ph.y * rho);
  }
  cs[j] = c;
  sn[j] = sv;
  col[j] = rjj;
  double2* gm = s.gamma + (int64_t)r * (s.m + 1);
  const double2 gj = gm[j];
  gm[j + 1] = make_double2(-(sv.x * gj.x + sv.y * gj.y), -(sv.x * gj.y - sv.y * gj.x));
  gm[j] = make_double2(c * gj.x, c * gj.y);
  s.k[r] = j + 1;
  const double res = hypot(gm[j + 1].x, gm[j + 1].y);
  const bool bad = !(isfinite(res) && isfinite(beta));
  const bool stop = bad || res <= s.thr[r] || beta <= 1e-14 * sqrt(w2) || j == s.m - 1;
  if (stop) {
    s.done[r] = 1;
    if (bad) s.k[r] = j;  // discard the step that produced a non-finite value
  }
  return !stop;
}

// Column j of the Hessenberg matrix from the Gram-Schmidt coefficients (CGS1 / CGS2)
// and the Givens step; scale = 1 / beta for the normalisation of the next vector.
__global__ void givens_kernel(GmresState s, int j, const double2* __restrict__ h1,
                              const double2* __restrict__ h2, const double2* __restrict__ hn, int pythag) {
  const int r = threadIdx.x;
  const int nrhs = s.nrhs;
  bool live = false;
  if (r < nrhs) {
    if (!s.done[r]) {
      double2* col = s.H + ((int64_t)r * s.m + j) * (s.m + 1);
      double w2 = 0.0, h2sq = 0.0;
      for (int i = 0; i <= j; ++i) {
        double2 v = h1[(int64_t)i * nrhs + r];
        if (h2 != nullptr) {
          const double2 u = h2[(int64_t)i * nrhs + r];
          h2sq += u.x * u.x + u.y * u.y;
          v.x += u.x;
          v.y += u.y;
        }
        col[i] = v;
        w2 += v.x * v.x + v.y * v.y;
      }
      const double beta2 = fmax(hn[(int64_t)(j + 1) * nrhs + r].x - (pythag ? h2sq : 0.0), 0.0);
      const double beta = sqrt(beta2);
      w2 += beta2;
      live = givens_step(s, r, j, col, beta, w2);
      s.scale[r] = live ? (beta > 0.0 ? 1.0 / beta : 0.0) : 0.0;
    } else {
      s.scale[r] = 0.0;
    }
  }
  const int any = __syncthreads_or(live);
  if (threadIdx.x == 0) *s.all_done = any ? 0 : 1;
}

// ---------------------------------------------------------------- delayed CGS2
//
// Classical Gram-Schmidt with the re-orthogonalisation delayed by one step, so that
// each Arnoldi step reads the basis twice instead of three times. The basis slots keep
// the once-orthogonalised candidates q~_0 .. q~_j (q~_0 = q_0 = r / ||r||); with the
// orthonormal basis Q they satisfy Q~_{j+1} = Q_{j+1} T_{j+1}, T upper triangular with
// columns [a_i; rho_i] (q~_i = Q_i a_i + rho_i q_i). Q is never formed. At step j, w = A q~_j:
//   pass A: e = Q~_{j+1}^H w, omega = ||w||^2;
//   coef2:  z = Q_{j+1}^H w = T^{-H} e (= [b; c], the projection on the final basis),
//           nu^2 = omega - |z|^2 (Pythagoras; nu only normalises the next candidate, its
//           error is absorbed one step later), g = T^{-1} z;
//   pass B: q~_{j+1} = (w - Q~_{j+1} g) / nu = (w - Q_{j+1} z) / nu, d = Q~_{j+1}^H (nu q~_{j+1}),
//           ||nu q~_{j+1}||^2;
//   coef1:  a_{j+1} = T^{-H} d / nu, rho_{j+1}^2 = ||q~_{j+1}||^2 - |a_{j+1}|^2 (T grows by a
//           column), and Hessenberg column j: A q_j = (A q~_j - A Q_j a_j) / rho_j with
//           q~_{j+1} = Q_{j+1} a_{j+1} + rho_{j+1} q_{j+1} gives
//           H_{l,j} = (z_l + nu a_{j+1,l} - (H_{:,<j} a_j)_l) / rho_j (l <= j), H_{j+1,j} = nu rho_{j+1} / rho_j
//           (H_{:,<j} the unrotated earlier columns), then its Givens step and the stop test,
//           before the next operator apply (finished rhs skip it).
// After the cycle x += Q_k y = Q~_k (T_k^{-1} y). One warp per rhs, lane l on basis index l
// (restart length <= 32); the triangular solves run over the lanes with shuffles.
struct DcgsState {
  double2* Hraw;    // [nrhs][m][m + 1] unrotated final columns
  double2* T;       // [nrhs][m + 1][m + 1] column-major: T[c][l], l <= c
  double2* z;       // [nrhs][m + 1] pending projection z of the current step
  double* nu;       // [nrhs]
  double2* g;       // [m + 1][nrhs] pass-B update coefficients
  unsigned* ctr;    // [2] live-rhs count and CTA ticket of the column kernel (0 between launches)
};

// One CTA (one warp) per rhs; the triangular factor and the Hessenberg columns are staged
// in shared memory, so that the sequential substitutions wait on shuffles, not on loads.
constexpr int kDcgsMaxM = 32;
constexpr int kDcgsLd = kDcgsMaxM + 1;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}
__device__ __forceinline__ double2 shfl2(double2 v, int src) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// Columns 0 .. n-1 of T (upper triangle) into Ts[c][l], reciprocals of the (real) diagonal.
__device__ __forceinline__ void stage_T(const double2* __restrict__ T, int ldt, int n, int lane,
                                        double2 (*Ts)[kDcgsLd], double* inv_d) {
#pragma unroll 4
  for (int c = 0; c < n; ++c)
    if (lane <= c) Ts[c][lane] = T[(int64_t)c * ldt + lane];
  __syncwarp();
  if (lane < n) inv_d[lane] = 1.0 / Ts[lane][lane].x;
  __syncwarp();
}

// x = T^{-H} v for the n x n leading block (lane l holds v_l on entry, x_l on return):
// forward substitution with the lower-triangular T^H, (T^H)_{l,i} = conj(T_{i,l}).
__device__ double2 solve_TH(const double2 (*Ts)[kDcgsLd], const double* inv_d, int n, int lane, double2 v) {
  for (int i = 0; i < n; ++i) {
    double2 xi = shfl2(v, i);
    const double di = inv_d[i];
    xi.x *= di;
    xi.y *= di;
    if (lane == i) {
      v = xi;
    } else if (lane > i && lane < n) {
      const double2 t = Ts[lane][i];  // T_{i,lane}
      v.x -= t.x * xi.x + t.y * xi.y;
      v.y -= t.x * xi.y - t.y * xi.x;
    }
  }
  return v;
}
// x = T^{-1} v (back substitution with the upper-triangular T).
__device__ double2 solve_T(const double2 (*Ts)[kDcgsLd], const double* inv_d, int n, int lane, double2 v) {
  for (int i = n - 1; i >= 0; --i) {
    double2 xi = shfl2(v, i);
    const double di = inv_d[i];
    xi.x *= di;
    xi.y *= di;
    if (lane == i) {
      v = xi;
    } else if (lane < i) {
      const double2 t = Ts[i][lane];  // T_{lane,i}
      v.x -= t.x * xi.x - t.y * xi.y;
      v.y -= t.x * xi.y + t.y * xi.x;
    }
  }
  return v;
}

// coef2 after pass A of step j (e: Q~_{j+1}^H w in slots 0 .. j, ||w||^2 in slot j + 1).
__global__ void __launch_bounds__(32) dcgs_coef2_kernel(GmresState s, DcgsState d, int j,
                                                        const double2* __restrict__ e) {
  __shared__ double2 Ts[kDcgsMaxM][kDcgsLd];
  __shared__ double inv_d[kDcgsMaxM];
  const int lane = threadIdx.x, r = blockIdx.x;
  const int nrhs = s.nrhs, m = s.m, n = j + 1;
  double2* T = d.T + (int64_t)r * (m + 1) * (m + 1);
  if (s.done[r]) {  // finished rhs: next candidate 0
    if (lane <= j) d.g[(int64_t)lane * nrhs + r] = make_double2(0.0, 0.0);
    if (lane == 0) s.scale[r] = 0.0;
    return;
  }
  if (j == 0) {
    if (lane == 0) {
      T[0] = make_double2(1.0, 0.0);
      Ts[0][0] = make_double2(1.0, 0.0);
      inv_d[0] = 1.0;
    }
    __syncwarp();
  } else {
    stage_T(T, m + 1, n, lane, Ts, inv_d);
  }
  const double2 v = lane <= j ? e[(int64_t)lane * nrhs + r] : make_double2(0.0, 0.0);
  const double2 z = solve_TH(Ts, inv_d, n, lane, v);
  const double zsq = warp_sum(lane <= j ? z.x * z.x + z.y * z.y : 0.0);
  const double omega = e[(int64_t)(j + 1) * nrhs + r].x;
  const double nu = sqrt(fmax(omega - zsq, 1e-12 * omega));
  const double2 g = solve_T(Ts, inv_d, n, lane, z);
  if (lane <= j) {
    d.z[(int64_t)r * (m + 1) + lane] = z;
    d.g[(int64_t)lane * nrhs + r] = g;
  }
  if (lane == 0) {
    d.nu[r] = nu;
    const bool ok = isfinite(nu) && nu > 0.0;
    s.scale[r] = ok ? 1.0 / nu : 0.0;
    if (!ok) s.done[r] = 1;
  }
}

// coef1 after pass B of step j (dd: Q~_{j+1}^H (nu q~_{j+1}) in slots 0 .. j, the norm in
// slot j + 1): the new column of T, final Hessenberg column j and its Givens step. The last
// CTA to finish sets the all-finished flag from the count of live rhs.
__global__ void __launch_bounds__(32) dcgs_coef1_kernel(GmresState s, DcgsState d, int j,
                                                        const double2* __restrict__ dd) {
  __shared__ double2 Ts[kDcgsMaxM][kDcgsLd];
  __shared__ double2 Hs[kDcgsMaxM][kDcgsLd];
  __shared__ double inv_d[kDcgsMaxM];
  __shared__ double cs_s[kDcgsMaxM];
  __shared__ double2 sn_s[kDcgsMaxM];
  const int lane = threadIdx.x, r = blockIdx.x;
  const int nrhs = s.nrhs, m = s.m, n = j + 1;
  int go = 0;
  if (!s.done[r]) {
    double2* T = d.T + (int64_t)r * (m + 1) * (m + 1);
    const double2* Hr = d.Hraw + (int64_t)r * m * (m + 1);
    if (lane < j) {  // the earlier rotations, for the Givens step below
      cs_s[lane] = s.cs[(int64_t)r * m + lane];
      sn_s[lane] = s.sn[(int64_t)r * m + lane];
    }
    stage_T(T, m + 1, n, lane, Ts, inv_d);
#pragma unroll 4
    for (int k = 0; k < j; ++k)  // column k has rows 0 .. k + 1
      if (lane <= k + 1) Hs[k][lane] = Hr[(int64_t)k * (m + 1) + lane];
    __syncwarp();
    const double nu = d.nu[r];
    const double inv_nu = nu > 0.0 ? 1.0 / nu : 0.0;
    double2 v = lane <= j ? dd[(int64_t)lane * nrhs + r] : make_double2(0.0, 0.0);
    v.x *= inv_nu;
    v.y *= inv_nu;
    const double2 an = solve_TH(Ts, inv_d, n, lane, v);  // a_{j+1}
    const double asq = warp_sum(lane <= j ? an.x * an.x + an.y * an.y : 0.0);
    const double alpha = dd[(int64_t)(j + 1) * nrhs + r].x * inv_nu * inv_nu;
    const double rho_n = sqrt(fmax(alpha - asq, 0.0));
    const double inv_rho_j = inv_d[j];  // 1 / rho_j
    double2 h = make_double2(0.0, 0.0);
    if (lane <= j) {
      const double2 zl = d.z[(int64_t)r * (m + 1) + lane];
      h = make_double2(zl.x + nu * an.x, zl.y + nu * an.y);
      for (int k = (lane > 0 ? lane - 1 : 0); k < j; ++k) {
        const double2 hk = Hs[k][lane];
        const double2 ak = Ts[j][k];  // a_j = T[0 .. j-1, j]
        h.x -= hk.x * ak.x - hk.y * ak.y;
        h.y -= hk.x * ak.y + hk.y * ak.x;
      }
      h.x *= inv_rho_j;
      h.y *= inv_rho_j;
      d.Hraw[((int64_t)r * m + j) * (m + 1) + lane] = h;
      Hs[j][lane] = h;
    }
    const double beta = nu * rho_n * inv_rho_j;
    const double w2 = warp_sum(h.x * h.x + h.y * h.y) + beta * beta;
    // the new column of T (used from the next step on)
    if (lane <= j) T[(int64_t)(j + 1) * (m + 1) + lane] = an;
    __syncwarp();
    if (lane == 0) {
      T[(int64_t)(j + 1) * (m + 1) + j + 1] = make_double2(rho_n, 0.0);
      d.Hraw[((int64_t)r * m + j) * (m + 1) + j + 1] = make_double2(beta, 0.0);
      // rotate the shared-memory copy of the column, then store it
      go = givens_step(s, r, j, Hs[j], beta, w2, cs_s, sn_s) && rho_n > 0.0 && isfinite(rho_n);
      if (!go) s.done[r] = 1;
    }
    __syncwarp();
    if (lane <= j) s.H[((int64_t)r * m + j) * (m + 1) + lane] = Hs[j][lane];
  }
  if (lane == 0) {
    if (go) atomicAdd(&d.ctr[0], 1u);
    __threadfence();
    const unsigned ticket = atomicAdd(&d.ctr[1], 1u);
    if (ticket == gridDim.x - 1) {
      __threadfence();
      const unsigned live = atomicAdd(&d.ctr[0], 0u);
      *s.all_done = live ? 0 : 1;
      d.ctr[0] = 0u;
      d.ctr[1] = 0u;
    }
  }
}

// After the back substitution: y <- T_k^{-1} y per rhs (x += Q~_k T_k^{-1} y).
__global__ void __launch_bounds__(32) dcgs_y_kernel(GmresState s, DcgsState d) {
  __shared__ double2 Ts[kDcgsMaxM][kDcgsLd];
  __shared__ double inv_d[kDcgsMaxM];
  const int lane = threadIdx.x, r = blockIdx.x;
  const int nrhs = s.nrhs, m = s.m;
  const int k = s.k[r];
  if (k == 0) return;
  stage_T(d.T + (int64_t)r * (m + 1) * (m + 1), m + 1, k, lane, Ts, inv_d);
  double2 v = lane < k ? s.y[(int64_t)lane * nrhs + r] : make_double2(0.0, 0.0);
  v = solve_T(Ts, inv_d, k, lane, v);
  if (lane < k) s.y[(int64_t)lane * nrhs + r] = v;
}

// Back substitution R y = gamma per rhs; y stored [m][nrhs]; kmax = max_r k_r.
__global__ void backsub_kernel(GmresState s) {
  const int r = threadIdx.x;
  int kr = 0;
  if (r < s.nrhs) {
    kr = s.k[r];
    double2 yv[64];
    for (int i = kr - 1; i >= 0; --i) {
      double2 acc = s.gamma[(int64_t)r * (s.m + 1) + i];
      for (int l = i + 1; l < kr; ++l) {
        const double2 h = s.H[((int64_t)r * s.m + l) * (s.m + 1) + i];
        acc.x -= h.x * yv[l].x - h.y * yv[l].y;
        acc.y -= h.x * yv[l].y + h.y * yv[l].x;
      }
      const double2 d = s.H[((int64_t)r * s.m + i) * (s.m + 1) + i];
      const double den = d.x * d.x + d.y * d.y;
      yv[i] = den > 0.0 ? make_double2((acc.x * d.x + acc.y * d.y) / den, (acc.y * d.x - acc.x * d.y) / den)
                        : make_double2(0.0, 0.0);
    }
    for (int i = 0; i < s.m; ++i) s.y[(int64_t)i * s.nrhs + r] = i < kr ? yv[i] : make_double2(0, 0);
  }
  __shared__ int kmax_s;
  if (threadIdx.x == 0) kmax_s = 0;
  __syncthreads();
  if (r < s.nrhs) atomicMax(&kmax_s, kr);
  __syncthreads();
  if (threadIdx.x == 0) *s.kmax = kmax_s;
}

__global__ void combine_h_kernel(int nvec, int nrhs, const double2* h1, const double2* h2,
                                 const double2* hn, double2* h, double* hnorm) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nvec * nrhs) {
    double2 v = h1[q];
    if (h2) { v.x += h2[q].x; v.y += h2[q].y; }
    h[q] = v;
  }
  if (q < nrhs) hnorm[q] = sqrt(fmax(hn[(int64_t)nvec * nrhs + q].x, 0.0));
}

static int round_threads(int n) { return ((n + 31) / 32) * 32; }

cudaError_t launch_cycle_init(const GmresState& s, const double* beta0, cudaStream_t stream) {
  cycle_init_kernel<<<1, round_threads(s.nrhs), 0, stream>>>(s, beta0);
  return cudaGetLastError();
}
cudaError_t launch_givens(const GmresState& s, int j, const void* h1, const void* h2, const void* hn,
                          bool pythag, cudaStream_t stream) {
  givens_kernel<<<1, round_threads(s.nrhs), 0, stream>>>(s, j, (const double2*)h1, (const double2*)h2,
                                                         (const double2*)hn, pythag ? 1 : 0);
  return cudaGetLastError();
}
static cudaError_t launch_dcgs_coef1(const GmresState& s, const DcgsState& d, int j, const void* dd,
                                     cudaStream_t stream) {
  dcgs_coef1_kernel<<<s.nrhs, 32, 0, stream>>>(s, d, j, (const double2*)dd);
  return cudaGetLastError();
}
static cudaError_t launch_dcgs_coef2(const GmresState& s, const DcgsState& d, int j, const void* e,
                                     cudaStream_t stream) {
  dcgs_coef2_kernel<<<s.nrhs, 32, 0, stream>>>(s, d, j, (const double2*)e);
  return cudaGetLastError();
}
static cudaError_t launch_dcgs_y(const GmresState& s, const DcgsState& d, cudaStream_t stream) {
  dcgs_y_kernel<<<s.nrhs, 32, 0, stream>>>(s, d);
  return cudaGetLastError();
}
cudaError_t launch_backsub(const GmresState& s, cudaStream_t stream) {
  backsub_kernel<<<1, round_threads(s.nrhs), 0, stream>>>(s);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ solver pieces

struct SolveBufs {
  bool f64_inner;
  bool bf16;            // basis stored as BF16 pairs, FP32 arithmetic, new vector in w32
  void* w32;            // FP32 buffer of the vector being orthogonalised (bf16 mode)
  int nrhs, m;
  int64_t n_sys;        // complex elements of the system vector
  size_t inner_bytes;   // bytes per inner basis vector
  void* basis;          // (m + 1) inner vectors
  void* tmp_even_in;    // Schur scratch, inner precision
  void* tmp_even_64;    // Schur scratch, FP64
  void* partials;
  void* h1;             // [m + 1][nrhs] double2 each
  void* h2;
  void* hn;
  GmresState st;
  BlasPlan plan;
  int ortho;            // 0: CGS1, 1: CGS2 (three passes), 2: delayed CGS2 (two passes)
  DcgsState dc;         // ortho == 2
};

// Gram-Schmidt of w = basis[j+1] against basis[0..j], the Givens step, and the
// normalisation v_{j+1} = w / beta (0 for rhs whose cycle has finished).
//   CGS2: h1 = V^H w; w' = w - V h1 with h2 = V^H w' and ||w'||^2; Givens with
//         beta^2 = ||w'||^2 - |h2|^2 (Pythagoras: V h2 is orthogonal to the final w);
//         v_{j+1} = (w' - V h2) / beta in the same pass.
//   CGS1: h1 = V^H w; w' = w - V h1 with ||w'||^2; Givens; v_{j+1} = w' / beta.
// The profiled Gram-Schmidt time covers all of it (the one-CTA Givens kernel included).
static lqcd_status arnoldi_ortho(const SolveBufs& b, int j, bool reorth, cudaEvent_t ev_gs_end, cudaStream_t s) {
  const int nvec = j + 1;
  char* base = (char*)b.basis;
  void* next = base + (size_t)(j + 1) * b.inner_bytes;
  void* w = b.bf16 ? b.w32 : next;
  const int64_t vstride = b.n_sys;
  const int* skip = b.st.all_done;
  if (b.ortho == 2) {
    // delayed CGS2: pass A (dots + norm of w), coefficients, pass B (the next candidate, its
    // dots and norm), then the final column j and its Givens step
    LQCD_CUDA(launch_gs_pass(false, b.plan, b.n_sys, nvec, b.basis, vstride, w, nullptr, false, true, true,
                             b.partials, b.h1, skip, s, nullptr, b.bf16),
              "dcgs pass A");
    LQCD_CUDA(launch_dcgs_coef2(b.st, b.dc, j, b.h1, s), "dcgs coefficients");
    LQCD_CUDA(launch_gs_pass(false, b.plan, b.n_sys, nvec, b.basis, vstride, w, b.dc.g, true, true, true,
                             b.partials, b.h2, skip, s, b.st.scale, b.bf16, b.bf16 ? next : nullptr),
              "dcgs pass B");
    LQCD_CUDA(launch_dcgs_coef1(b.st, b.dc, j, b.h2, s), "dcgs column");
    if (ev_gs_end) LQCD_CUDA(cudaEventRecord(ev_gs_end, s), "event");
    return LQCD_OK;
  }
  LQCD_CUDA(launch_gs_pass(b.f64_inner, b.plan, b.n_sys, nvec, b.basis, vstride, w, nullptr, false, true,
                           false, b.partials, b.h1, skip, s, nullptr, b.bf16),
            "gs dots");
  if (reorth) {
    LQCD_CUDA(launch_gs_pass(b.f64_inner, b.plan, b.n_sys, nvec, b.basis, vstride, w, b.h1, true, true,
                             true, b.partials, b.h2, skip, s, nullptr, b.bf16),
              "gs update+dots+norm");
    LQCD_CUDA(launch_givens(b.st, j, b.h1, b.h2, b.h2, true, s), "givens");
    LQCD_CUDA(launch_gs_pass(b.f64_inner, b.plan, b.n_sys, nvec, b.basis, vstride, w, b.h2, true, false,
                             false, b.partials, nullptr, skip, s, b.st.scale, b.bf16, b.bf16 ? next : nullptr),
              "gs update+scale");
  } else {
    LQCD_CUDA(launch_gs_pass(b.f64_inner, b.plan, b.n_sys, nvec, b.basis, vstride, w, b.h1, true, false,
                             true, b.partials, b.hn, skip, s),
              "gs update+norm");
    LQCD_CUDA(launch_givens(b.st, j, b.h1, nullptr, b.hn, false, s), "givens");
    LQCD_CUDA(launch_scale_inplace(b.f64_inner, b.n_sys, b.nrhs, w, b.st.scale, skip, s), "scale");
  }
  if (ev_gs_end) LQCD_CUDA(cudaEventRecord(ev_gs_end, s), "event");
  return LQCD_OK;
}

struct Profile {
  bool on = false;
  std::vector<cudaEvent_t> ev;  // 4 per step: op start/end, gs start/end
  double op_ms = 0, gs_ms = 0;
  double op_bytes = 0, gs_bytes = 0;
  int op_n = 0, gs_n = 0;
  int used = 0;
};

// Algorithmic bytes (each operand moved once) of one operator apply on a packed block:
// full: (48 b + 144) s per site with clover, (48 b + 72) s without;
// Schur: (120 b + 432) s per odd site with clover, (120 b + 288) s without
// (s = bytes per real; spinors read/written once per pass, 18 reals per link,
// 72 reals per site block).
static double op_algorithmic_bytes(const lqcd_ctx_s* ctx, int op, bool f64, int nrhs, bool bf16 = false) {
  const double s = f64 ? 8.0 : 4.0;
  const bool clover = ctx->c_sw != 0.0;
  // links: 72 reals per site (full) or 288 per odd site (Schur) in the 18-real form; the
  // two-row forms read 12 reals per link (BF16 storage: 2 bytes each, expressed in units of s)
  double link_reals = op == LQCD_OP_FULL ? 72.0 : 288.0;
  if (!f64) {
    const int v = tuned_variant(ctx, false, nrhs, op);
    if (ctx->link_format == LQCD_LINKS_BF16) link_reals *= (12.0 * 2.0) / (18.0 * 4.0);
    else if (v >= 0 && dslash_variant(false, v).links == 1) link_reals *= 12.0 / 18.0;
  }
  const double fixed = (op == LQCD_OP_FULL ? (clover ? 72.0 : 0.0) : (clover ? 144.0 : 0.0)) + link_reals;
  if (bf16) {  // BF16 input read (2 bytes per real), FP32 intermediate and output
    if (op == LQCD_OP_FULL) return (double)ctx->g.V * (24.0 * nrhs * 2 + 24.0 * nrhs * 4 + fixed * 4);
    return (double)ctx->g.Vh * (2 * 24.0 * nrhs * 2 + 3 * 24.0 * nrhs * 4 + fixed * 4);
  }
  if (op == LQCD_OP_FULL) return (double)ctx->g.V * (48.0 * nrhs + fixed) * s;
  return (double)ctx->g.Vh * (120.0 * nrhs + fixed) * s;
}

// Algorithmic bytes of the Gram-Schmidt step with nvec basis vectors on n complex
// elements: the dot pass reads nvec + 1 vectors; each update pass reads nvec + 1
// and writes 1 (CGS2: two updates, the second one normalising; CGS1: one update
// and a separate normalisation that reads and writes w once more).
static double gs_algorithmic_bytes(int64_t n, int nvec, bool f64, int ortho, bool bf16 = false) {
  const double vb = (double)n * (bf16 ? 4.0 : (f64 ? 16.0 : 8.0));  // a basis vector
  const double vw = (double)n * (f64 ? 16.0 : 8.0);                  // w (FP32 for a BF16 basis)
  if (ortho == 2)  // delayed CGS2: two reads of the basis and w, one write of the next candidate
    return 2 * (nvec * vb + vw) + vb;
  if (bf16)  // CGS2 with a BF16 basis; the last pass writes the BF16 basis vector
    return (nvec * vb + vw) + (nvec * vb + 2 * vw) + (nvec * vb + vw + vb);
  const double dots = (nvec + 1) * vw, upd = (nvec + 2) * vw;
  return ortho == 1 ? dots + 2 * upd : dots + upd + 2 * vw;
}

static lqcd_status run_cycle_direct(lqcd_ctx ctx, const SolveBufs& b, int op, bool reorth, Profile* prof,
                                    cudaStream_t s) {
  char* base = (char*)b.basis;
  for (int j = 0; j < b.m; ++j) {
    void* vj = base + (size_t)j * b.inner_bytes;
    void* w = base + (size_t)(j + 1) * b.inner_bytes;
    if (prof->on) LQCD_CUDA(cudaEventRecord(prof->ev[4 * j + 0], s), "event");
    lqcd_status st = b.bf16 ? apply_operator_bf16in(ctx, op, b.nrhs, vj, b.w32, b.tmp_even_in, b.st.all_done, s)
                            : apply_operator(ctx, op, b.f64_inner, b.nrhs, vj, w, b.tmp_even_in, b.st.all_done, s);
    if (st != LQCD_OK) return st;
    if (prof->on) {
      LQCD_CUDA(cudaEventRecord(prof->ev[4 * j + 1], s), "event");
      LQCD_CUDA(cudaEventRecord(prof->ev[4 * j + 2], s), "event");
    }
    st = arnoldi_ortho(b, j, reorth, prof->on ? prof->ev[4 * j + 3] : nullptr, s);
    if (st != LQCD_OK) return st;
  }
  if (prof->on) prof->used = b.m;
  return LQCD_OK;
}

static lqcd_status run_cycle(lqcd_ctx ctx, const SolveBufs& b, int op, bool reorth, bool use_graph,
                             Profile* prof, cudaStream_t s) {
  // CUDA events recorded inside a graph do not time its kernel nodes, so a
  // profiled cycle is launched kernel by kernel.
  if (!use_graph || prof->on) return run_cycle_direct(ctx, b, op, reorth, prof, s);
  char key[256];
  snprintf(key, sizeof(key), "%d/%d/%d/%d/%d/%d/%d/%p/%p/%p/%p/%p/%lld", op, (int)b.f64_inner, (int)b.bf16, b.nrhs, b.m,
           (int)reorth, b.ortho, b.basis, b.w32, b.partials, (void*)b.st.H, (void*)b.dc.g, (long long)b.n_sys);
  if (ctx->cycle.exec == nullptr || ctx->cycle.key != key) {
    if (ctx->cycle.exec) {
      cudaGraphExecDestroy(ctx->cycle.exec);
      cudaGraphDestroy(ctx->cycle.graph);
      ctx->cycle.exec = nullptr;
      ctx->cycle.graph = nullptr;
    }
    if (!ctx->capture_stream)
      LQCD_CUDA(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking), "capture stream");
    LQCD_CUDA(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    Profile none;
    lqcd_status st = run_cycle_direct(ctx, b, op, reorth, &none, ctx->capture_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->capture_stream, &g);
    if (st != LQCD_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_error(e, "end capture");
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      return cuda_error(e, "graph instantiate");
    }
    ctx->cycle.graph = g;
    ctx->cycle.exec = ex;
    ctx->cycle.key = key;
  }
  LQCD_CUDA(cudaGraphLaunch(ctx->cycle.exec, s), "graph launch");
  return LQCD_OK;
}

// Accumulate the event times of the steps that ran (j < kmax: later steps were
// skipped on the device once every rhs had finished its cycle).
static void collect_profile(Profile* prof, int kmax, double op_bytes, int64_t n, bool f64, int ortho, bool bf16) {
  if (!prof->on) return;
  for (int j = 0; j < prof->used && j < kmax; ++j) {
    float a = 0.f, c = 0.f;
    if (cudaEventElapsedTime(&a, prof->ev[4 * j], prof->ev[4 * j + 1]) == cudaSuccess) {
      prof->op_ms += a;
      prof->op_n += 1;
      prof->op_bytes += op_bytes;
    }
    if (cudaEventElapsedTime(&c, prof->ev[4 * j + 2], prof->ev[4 * j + 3]) == cudaSuccess) {
      prof->gs_ms += c;
      prof->gs_n += 1;
      prof->gs_bytes += gs_algorithmic_bytes(n, j + 1, f64, ortho, bf16);
    }
  }
  prof->used = 0;
  cudaGetLastError();
}

}  // namespace lqcd


namespace lqcd {

// Pinned staging layout used by the solve (host side of the per-rhs scalars).
struct Staging {
  double rn2[2 * 256];      // reduced double2 norms (x, y)
  double beta0[256];
  double thr[256];
  int active[256];
  int kcycle[256];
  int wait_err;             // the streaming kernels' pipeline-wait flag
  double block_res[64];     // block GMRES: residual norm per rhs after the last step
  int block_flag;           // block GMRES: rank-deficient block met
};

// One lattice's batched-GMRES solve, split into the phases of a restart so that
// a single solve and a batch of solves on several lattices share the same code.
struct SolveJob {
  lqcd_ctx ctx = nullptr;
  lqcd_solve_params P;
  int nrhs = 0;
  const void* b = nullptr;
  void* x = nullptr;
  lqcd_solve_stats* stats = nullptr;
  cudaStream_t s = nullptr;
  std::chrono::steady_clock::time_point t0;
  bool eo = false, f64_inner = false, bf16 = false, reorth = true;
  int m = 0;
  int ortho_req = 1;
  double inner_tol = 0.0;
  int64_t n_full = 0, n_half = 0, n_sys = 0;
  size_t full64 = 0;
  void *b_can = nullptr, *x_can = nullptr, *b64 = nullptr, *x64 = nullptr, *r64 = nullptr, *t64 = nullptr;
  void *bhat = nullptr, *tmp64 = nullptr, *sys_b = nullptr, *sys_x = nullptr, *red_partials = nullptr;
  bool b_host = false, x_host = false;
  SolveBufs B;
  BlasPlan plan_full;
  double* d_beta0 = nullptr;
  Staging* hs = nullptr;
  Profile prof;
  std::vector<int> iters;
  std::vector<double> relres, bnorm;
  int restarts = 0;
  bool pending_k = false;
  bool finished = false;
  // nested refinement (FP32 / BF16 inner): inner restarts start from the FP32 residual
  // of the correction equation, r_outer - D (x - x_outer); an FP64 residual follows
  // each inner solve
  bool nested = false;
  bool outer_next = true;   // the next residual is the FP64 one
  bool last_outer = true;   // the residual being decided was the FP64 one
  int inner_cycles = 0;
  int outer_steps = 0;
  void *x_outer = nullptr, *r_outer = nullptr, *e32 = nullptr, *t32 = nullptr;
  std::vector<double> rn_prev;
  std::vector<char> active_outer, inner_done;
  long long nl = 0;  // kernel launches of this solve
  double op_bytes_inner = 0.0;
  lqcd_status result = LQCD_NOT_CONVERGED;
  // compaction of the active rhs (params.compact): the solve runs on nrhs columns of the
  // caller's nrhs0; col[k] is the caller's column of current column k, b_cur / x_cur the
  // FP64 packed full blocks of the current columns (b64 / x64, the caller's, before any
  // compaction). x64 keeps every caller column's latest solution.
  int nrhs0 = 0;
  std::vector<int> col;
  void *b_cur = nullptr, *x_cur = nullptr;
  std::vector<int> iters0;
  std::vector<double> bnorm0;
  int compactions = 0;

  lqcd_status setup(lqcd_ctx c, const lqcd_solve_params* params, int nr, const void* bb, void* xx,
                    lqcd_solve_stats* st_out, cudaStream_t stream);
  // buffers, plans and the system right-hand side for the current column count
  lqcd_status configure();
  // keep only the current columns listed in keep (at an FP64 restart)
  lqcd_status compact(const std::vector<int>& keep);
  lqcd_status enqueue_residual();
  // after the stream has been synchronised: *run = a cycle follows; with neither run
  // nor finished, the next residual (the FP64 one) is due before the next cycle
  lqcd_status decide(bool* run);
  lqcd_status enqueue_cycle(cudaStream_t cs, bool allow_graph);
  lqcd_status finish();
  // kernels of one restart cycle: cycle_init, v0, per step (operator, Gram-Schmidt
  // passes with their reductions, givens, normalisation), backsub (and the delayed-CGS2
  // change of basis of y), update
  long long cycle_launches() const { return 4 + (B.ortho == 2 ? 1 : 0) + (long long)m * ((eo ? 2 : 1) + 6); }
};

lqcd_status SolveJob::setup(lqcd_ctx c, const lqcd_solve_params* params, int nr, const void* bb, void* xx,
                            lqcd_solve_stats* st_out, cudaStream_t stream) {
  t0 = std::chrono::steady_clock::now();
  ctx = c; nrhs = nr; b = bb; x = xx; stats = st_out; s = stream;
  if (!ctx || !params || !b || !x) return set_error(LQCD_ERR_ARG, "lqcd_solve: null argument");
  P = *params;
  if (!ctx->have_gauge || !ctx->have_blocks)
    return set_error(LQCD_ERR_STATE, "lqcd_solve: set_gauge and set_clover must be called first");
  if (nrhs < 1 || nrhs > 64 || P.restart_len < 1 || P.restart_len > 64 || P.max_restarts < 1 ||
      !(P.tol > 0.0) || (P.op != LQCD_OP_FULL && P.op != LQCD_OP_SCHUR) ||
      (P.precision != LQCD_C64 && P.precision != LQCD_C128 && P.precision != LQCD_BF16S) ||
      (P.precision == LQCD_BF16S && nrhs > 32 && (nrhs % 2 != 0 || nrhs > 64)) ||
      (P.dagger != 0 && P.dagger != 1))
    return set_error(LQCD_ERR_ARG,
                     "lqcd_solve: bad parameters (nrhs 1..64, 1..32 for BF16 storage, restart_len 1..64, tol > 0)");
  if (P.block && (P.precision != LQCD_C64 || nrhs > 16))
    return set_error(LQCD_ERR_ARG, "lqcd_solve: block GMRES needs precision LQCD_C64 and at most 16 rhs");
  eo = P.op == LQCD_OP_SCHUR;
  f64_inner = P.precision == LQCD_C128;
  bf16 = P.precision == LQCD_BF16S;
  m = P.restart_len;
  reorth = P.reorth != 0 || bf16;
  ortho_req = P.reorth == 0 ? (bf16 ? 1 : 0) : (P.reorth == 2 ? 2 : 1);
  inner_tol = P.inner_tol > 0.0 ? P.inner_tol : (f64_inner ? 0.0 : 1e-4);
  n_full = (int64_t)packed_elems(ctx, LQCD_SITES_FULL, nrhs);
  n_half = n_full / 2;
  n_sys = eo ? n_half : n_full;
  full64 = (size_t)n_full * sizeof(double2);
  lqcd_status st;

  // ---------------- buffers
  b_can = (void*)b;
  x_can = x;
  b_host = !is_device_pointer(b);
  x_host = !is_device_pointer(x);
  if (b_host && (st = workspace(ctx, "solve_b_can", full64, &b_can)) != LQCD_OK) return st;
  if (x_host && (st = workspace(ctx, "solve_x_can", full64, &x_can)) != LQCD_OK) return st;
  if ((st = workspace(ctx, "solve_b64", full64, &b64)) != LQCD_OK) return st;
  if ((st = workspace(ctx, "solve_x64", full64, &x64)) != LQCD_OK) return st;
  if ((st = workspace(ctx, "solve_r64", full64, &r64)) != LQCD_OK) return st;
  if ((st = workspace(ctx, "solve_t64", full64, &t64)) != LQCD_OK) return st;
  if (eo) {
    if ((st = workspace(ctx, "solve_bhat", (size_t)n_half * sizeof(double2), &bhat)) != LQCD_OK) return st;
    if ((st = workspace(ctx, "schur_tmp64", (size_t)n_half * sizeof(double2), &tmp64)) != LQCD_OK) return st;
  }
  B.f64_inner = f64_inner;
  B.bf16 = bf16;
  B.w32 = nullptr;
  B.nrhs = nrhs;
  B.m = m;
  B.n_sys = n_sys;
  B.inner_bytes = (size_t)n_sys * (f64_inner ? sizeof(double2) : (bf16 ? sizeof(__nv_bfloat162) : sizeof(float2)));
  if ((st = workspace(ctx, "solve_basis", B.inner_bytes * (m + 1), &B.basis)) != LQCD_OK) return st;
  if (bf16 && (st = workspace(ctx, "solve_w32", (size_t)n_sys * sizeof(float2), &B.w32)) != LQCD_OK) return st;
  B.tmp_even_in = nullptr;
  if (eo) {
    if (f64_inner) B.tmp_even_in = tmp64;
    else if ((st = workspace(ctx, "schur_tmp32", (size_t)n_half * sizeof(float2), &B.tmp_even_in)) != LQCD_OK)
      return st;
  }
  nested = !f64_inner && !P.block;   // block GMRES: one block cycle per FP64 residual
  if (nested) {
    if ((st = workspace(ctx, "solve_x_outer", (size_t)n_sys * sizeof(double2), &x_outer)) != LQCD_OK) return st;
    if ((st = workspace(ctx, "solve_r_outer", (size_t)n_sys * sizeof(double2), &r_outer)) != LQCD_OK) return st;
    if ((st = workspace(ctx, "solve_e32", (size_t)n_sys * sizeof(float2), &e32)) != LQCD_OK) return st;
    if ((st = workspace(ctx, "solve_t32", (size_t)n_sys * sizeof(float2), &t32)) != LQCD_OK) return st;
  }
  if ((st = workspace(ctx, "solve_beta0", sizeof(double) * nrhs, (void**)&d_beta0)) != LQCD_OK) return st;
  if ((st = pinned_staging(ctx, sizeof(Staging), (void**)&hs)) != LQCD_OK) return st;
  prof.on = P.profile != 0;
  if (prof.on) {
    if (ctx->prof_events.empty()) {
      ctx->prof_events.resize(4 * 64);
      for (auto& e : ctx->prof_events) LQCD_CUDA(cudaEventCreate(&e), "event create");
    }
    prof.ev = ctx->prof_events;
  }

  // ---------------- inputs
  if (b_host) LQCD_CUDA(cudaMemcpyAsync(b_can, b, full64, cudaMemcpyHostToDevice, s), "upload b");
  if ((st = lqcd_pack(ctx, LQCD_C128, LQCD_SITES_FULL, nrhs, b_can, b64, s)) != LQCD_OK) return st;
  const int log_s = layout_for(ctx, nrhs).log_s;
  // adjoint system: D^dagger x = b is solved as D y = gamma5 b, x = gamma5 y
  if (P.dagger) LQCD_CUDA(launch_gamma5_packed(n_full, nrhs, log_s, b64, s), "gamma5 b");
  if (P.x0_given) {
    if (x_host) LQCD_CUDA(cudaMemcpyAsync(x_can, x, full64, cudaMemcpyHostToDevice, s), "upload x0");
    if ((st = lqcd_pack(ctx, LQCD_C128, LQCD_SITES_FULL, nrhs, x_can, x64, s)) != LQCD_OK) return st;
    if (P.dagger) LQCD_CUDA(launch_gamma5_packed(n_full, nrhs, log_s, x64, s), "gamma5 x0");
  } else {
    LQCD_CUDA(cudaMemsetAsync(x64, 0, full64, s), "zero x");
  }
  plan_full = blas_plan(n_full, nrhs, ctx->num_sms);
  if ((st = workspace(ctx, "solve_partials_full", sizeof(double2) * (size_t)nrhs * plan_full.blocks,
                      &red_partials)) != LQCD_OK)
    return st;
  if ((st = workspace(ctx, "solve_hn", sizeof(double2) * (size_t)(m + 1) * nrhs, &B.hn)) != LQCD_OK) return st;
  LQCD_CUDA(launch_norm2(true, plan_full, n_full, b64, red_partials, B.hn, s), "norm b");
  nl += (P.x0_given ? 2 : 1) + 2;  // packs, norm + reduction
  LQCD_CUDA(cudaMemcpyAsync(hs->rn2, B.hn, sizeof(double2) * nrhs, cudaMemcpyDeviceToHost, s), "read norm b");
  LQCD_CUDA(cudaStreamSynchronize(s), "sync");
  bnorm0.assign(nrhs, 0.0);
  for (int r = 0; r < nrhs; ++r) {
    bnorm0[r] = std::sqrt(hs->rn2[2 * r]);
    if (!std::isfinite(bnorm0[r]))
      return set_error(LQCD_ERR_NONFINITE, "lqcd_solve: right-hand side %d is not finite", r);
  }
  nrhs0 = nrhs;
  col.resize(nrhs);
  for (int r = 0; r < nrhs; ++r) col[r] = r;
  iters0.assign(nrhs, 0);
  b_cur = b64;
  x_cur = x64;
  return configure();
}

lqcd_status SolveJob::configure() {
  lqcd_status st;
  n_full = (int64_t)packed_elems(ctx, LQCD_SITES_FULL, nrhs);
  n_half = n_full / 2;
  n_sys = eo ? n_half : n_full;
  B.nrhs = nrhs;
  B.n_sys = n_sys;
  B.inner_bytes = (size_t)n_sys * (f64_inner ? sizeof(double2) : (bf16 ? sizeof(__nv_bfloat162) : sizeof(float2)));
  rn_prev.assign(nrhs, 0.0);
  active_outer.assign(nrhs, 0);
  inner_done.assign(nrhs, 1);
  B.plan = blas_plan(n_sys, nrhs, ctx->num_sms);
  B.plan.wait_flag = wait_flag(ctx);
  // delayed CGS2 needs the streaming Gram-Schmidt kernel for every basis size (FP32 or
  // BF16 basis) and restart length <= 32 (one warp per rhs in the coefficient kernels); otherwise CGS2
  B.ortho = ortho_req;
  if (B.ortho == 2 && (f64_inner || m > kDcgsMaxM ||
                       !(bf16 ? gs_stream_passes_supported_bf16(B.plan, n_sys, m)
                              : gs_stream_passes_supported_f32(B.plan, n_sys, m))))
    B.ortho = 1;
  memset(&B.dc, 0, sizeof(B.dc));
  if (B.ortho == 2) {
    const size_t dpiece[6] = {sizeof(double2) * (size_t)nrhs * m * (m + 1),
                              sizeof(double2) * (size_t)nrhs * (m + 1) * (m + 1),
                              sizeof(double2) * (size_t)nrhs * (m + 1), sizeof(double) * nrhs,
                              sizeof(double2) * (size_t)(m + 1) * nrhs, 2 * sizeof(unsigned)};
    size_t dbytes = 0;
    for (size_t q : dpiece) dbytes += (q + 255) & ~(size_t)255;
    void* dmem;
    if ((st = workspace(ctx, "solve_dcgs", dbytes, &dmem)) != LQCD_OK) return st;
    char* p = (char*)dmem;
    int next = 0;
    auto take = [&]() { void* q = p; p += (dpiece[next++] + 255) & ~(size_t)255; return q; };
    B.dc.Hraw = (double2*)take();
    B.dc.T = (double2*)take();
    B.dc.z = (double2*)take();
    B.dc.nu = (double*)take();
    B.dc.g = (double2*)take();
    B.dc.ctr = (unsigned*)take();
    LQCD_CUDA(cudaMemsetAsync(B.dc.ctr, 0, 2 * sizeof(unsigned), s), "dcgs counters");
  }
  const size_t hb = sizeof(double2) * (size_t)(m + 1) * nrhs;
  if ((st = workspace(ctx, "solve_partials", hb * B.plan.blocks, &B.partials)) != LQCD_OK) return st;
  if ((st = workspace(ctx, "solve_h1", hb, &B.h1)) != LQCD_OK) return st;
  if ((st = workspace(ctx, "solve_h2", hb, &B.h2)) != LQCD_OK) return st;
  if ((st = workspace(ctx, "solve_hn", hb, &B.hn)) != LQCD_OK) return st;
  // small per-rhs state, one allocation carved into 256-byte aligned pieces
  const size_t piece[12] = {sizeof(double2) * (size_t)nrhs * m * (m + 1), sizeof(double) * (size_t)nrhs * m,
                            sizeof(double2) * (size_t)nrhs * m, sizeof(double2) * (size_t)nrhs * (m + 1),
                            sizeof(double2) * (size_t)m * nrhs, sizeof(double) * nrhs, sizeof(double) * nrhs,
                            sizeof(int) * nrhs, sizeof(int) * nrhs, sizeof(int) * nrhs, sizeof(int), sizeof(int)};
  size_t small_bytes = 0;
  for (size_t q : piece) small_bytes += (q + 255) & ~(size_t)255;
  void* small;
  if ((st = workspace(ctx, "solve_small", small_bytes, &small)) != LQCD_OK) return st;
  {
    char* p = (char*)small;
    int next = 0;
    auto take = [&]() { void* q = p; p += (piece[next++] + 255) & ~(size_t)255; return q; };
    B.st.m = m;
    B.st.nrhs = nrhs;
    B.st.H = (double2*)take();
    B.st.cs = (double*)take();
    B.st.sn = (double2*)take();
    B.st.gamma = (double2*)take();
    B.st.y = (double2*)take();
    B.st.thr = (double*)take();
    B.st.scale = (double*)take();
    B.st.active = (int*)take();
    B.st.done = (int*)take();
    B.st.k = (int*)take();
    B.st.all_done = (int*)take();
    B.st.kmax = (int*)take();
  }
  bnorm.assign(nrhs, 0.0);
  for (int r = 0; r < nrhs; ++r) bnorm[r] = bnorm0[col[r]];
  sys_b = b_cur;
  sys_x = x_cur;
  if (eo) {
    if ((st = schur_prepare(ctx, true, nrhs, b_cur, bhat, tmp64, s)) != LQCD_OK) return st;
    sys_b = bhat;
    sys_x = (char*)x_cur + (size_t)n_half * sizeof(double2);
    nl += 2;
  }
  iters.assign(nrhs, 0);
  relres.assign(nrhs, 0.0);
  op_bytes_inner = op_algorithmic_bytes(ctx, P.op, f64_inner, nrhs, bf16);
  return LQCD_OK;
}

lqcd_status SolveJob::compact(const std::vector<int>& keep) {
  const int n2 = (int)keep.size();
  const int64_t V = ctx->g.V;
  const PackedLayout L0 = layout_for(ctx, nrhs0), Lc = layout_for(ctx, nrhs), L2 = layout_for(ctx, n2);
  ColumnMap mp;
  if (x_cur != x64) {  // the caller's block gets the latest solution of every current column
    for (int k = 0; k < nrhs; ++k) mp.col[k] = col[k];
    LQCD_CUDA(launch_repack_columns(V, Lc, L0, mp, true, x_cur, x64, s), "compaction scatter x");
  }
  std::vector<int> next(n2);
  for (int k = 0; k < n2; ++k) next[k] = mp.col[k] = col[keep[k]];
  const size_t bytes2 = (size_t)packed_elems(ctx, LQCD_SITES_FULL, n2) * sizeof(double2);
  lqcd_status st;
  void *bc, *xc;
  if ((st = workspace(ctx, "solve_b_compact", bytes2, &bc)) != LQCD_OK) return st;
  if ((st = workspace(ctx, "solve_x_compact", bytes2, &xc)) != LQCD_OK) return st;
  LQCD_CUDA(launch_repack_columns(V, L0, L2, mp, false, b64, bc, s), "compaction gather b");
  LQCD_CUDA(launch_repack_columns(V, L0, L2, mp, false, x64, xc, s), "compaction gather x");
  nl += (x_cur != x64 ? 1 : 0) + 2;
  for (int k = 0; k < nrhs; ++k) iters0[col[k]] += iters[k];
  col = next;
  nrhs = n2;
  b_cur = bc;
  x_cur = xc;
  ++compactions;
  return configure();
}

// The residual of the next restart and its norms, copied to the pinned staging area:
// the FP64 true residual r = b - D x (then, nested, x_outer = x and r_outer = r), or
// (nested, inner restart) r = r_outer - D_32 fl32(x - x_outer) with the FP32 operator.
lqcd_status SolveJob::enqueue_residual() {
  lqcd_status st;
  last_outer = !nested || outer_next;
  if (last_outer) {
    if ((st = apply_operator(ctx, P.op, true, nrhs, sys_x, t64, tmp64, nullptr, s)) != LQCD_OK) return st;
    LQCD_CUDA(launch_sub_norm(B.plan, n_sys, sys_b, t64, r64, B.partials, B.hn, s), "residual");
    nl += eo ? 4 : 3;  // FP64 operator + residual kernel + reduction
    if (nested) {
      LQCD_CUDA(cudaMemcpyAsync(x_outer, sys_x, (size_t)n_sys * sizeof(double2), cudaMemcpyDeviceToDevice, s),
                "save x");
      LQCD_CUDA(cudaMemcpyAsync(r_outer, r64, (size_t)n_sys * sizeof(double2), cudaMemcpyDeviceToDevice, s),
                "save r");
    }
  } else {
    LQCD_CUDA(launch_diff_to_f32(n_sys, sys_x, x_outer, e32, s), "correction");
    if ((st = apply_operator(ctx, P.op, false, nrhs, e32, t32, B.tmp_even_in, nullptr, s)) != LQCD_OK) return st;
    LQCD_CUDA(launch_sub_norm(B.plan, n_sys, r_outer, t32, r64, B.partials, B.hn, s, true), "inner residual");
    nl += eo ? 5 : 4;  // difference, FP32 operator, residual kernel + reduction
  }
  LQCD_CUDA(cudaMemcpyAsync(hs->rn2, B.hn, sizeof(double2) * nrhs, cudaMemcpyDeviceToHost, s), "read rn");
  hs->wait_err = 0;
  if (B.plan.wait_flag)
    LQCD_CUDA(cudaMemcpyAsync(&hs->wait_err, B.plan.wait_flag, sizeof(int), cudaMemcpyDeviceToHost, s), "read flag");
  return LQCD_OK;
}

// Host decision of one restart (the residual norms have arrived). After the FP64
// residual: retire the rhs that meet tol, set each cycle threshold from it. After
// an inner residual: an rhs ends its inner solve when the residual reaches the
// threshold, no longer decreases (less than 10% per cycle: the FP32 operator's
// rounding floor) or after kMaxInner cycles; when all have, the FP64 residual is due.
lqcd_status SolveJob::decide(bool* run) {
  constexpr int kMaxInner = 16;
  *run = false;
  if (pending_k) {
    int kmax = 0;
    for (int r = 0; r < nrhs; ++r) {
      iters[r] += hs->kcycle[r];
      kmax = std::max(kmax, hs->kcycle[r]);
    }
    collect_profile(&prof, kmax, op_bytes_inner, n_sys, f64_inner, B.ortho, bf16);
  }
  pending_k = false;
  if (hs->wait_err != 0)
    return set_error(LQCD_ERR_CUDA, "lqcd_solve: a Gram-Schmidt pipeline wait timed out (device flag %d)",
                     hs->wait_err);
  int n_active = 0;
  if (last_outer) {
    ++outer_steps;
    for (int r = 0; r < nrhs; ++r) {
      const double rn = std::sqrt(hs->rn2[2 * r]);
      if (!std::isfinite(rn))
        return set_error(LQCD_ERR_NONFINITE, "lqcd_solve: residual of rhs %d is not finite", r);
      relres[r] = bnorm[r] > 0.0 ? rn / bnorm[r] : 0.0;
      const bool act = bnorm[r] > 0.0 && rn > P.tol * bnorm[r];
      active_outer[r] = act ? 1 : 0;
      inner_done[r] = act ? 0 : 1;
      rn_prev[r] = rn;
      hs->active[r] = act ? 1 : 0;
      hs->beta0[r] = act ? rn : 1.0;
      // cycle target: half the tolerance (so the true residual, which the Arnoldi
      // estimate approximates, lands below tol), or the inner relative reduction
      double thr = 0.5 * P.tol * bnorm[r];
      if (inner_tol > 0.0) thr = std::max(thr, inner_tol * rn);
      hs->thr[r] = thr;
      n_active += act;
    }
    if (n_active == 0) {
      result = LQCD_OK;
      finished = true;
      return LQCD_OK;
    }
    if (restarts >= P.max_restarts) {
      finished = true;
      return LQCD_OK;
    }
    // (block GMRES always removes converged rhs: their near-zero residual columns would make
    // the block's Gram matrix ill-conditioned)
    if ((P.compact || P.block) && nrhs - n_active >= (P.block ? 1 : std::max(1, nrhs / 8))) {
      // retire the converged rhs from the block: the solve continues on the active
      // columns only, so the operator and Gram-Schmidt move fewer bytes; the FP64
      // residual of the compacted block is computed next
      std::vector<int> keep;
      for (int r = 0; r < nrhs; ++r)
        if (active_outer[r]) keep.push_back(r);
      lqcd_status st = compact(keep);
      if (st != LQCD_OK) return st;
      outer_next = true;
      return LQCD_OK;
    }
    outer_next = false;
    inner_cycles = 0;
  } else {
    ++inner_cycles;
    for (int r = 0; r < nrhs; ++r) {
      hs->active[r] = 0;
      hs->beta0[r] = 1.0;
      if (!active_outer[r] || inner_done[r]) continue;
      const double rn = std::sqrt(hs->rn2[2 * r]);
      if (!std::isfinite(rn))
        return set_error(LQCD_ERR_NONFINITE, "lqcd_solve: inner residual of rhs %d is not finite", r);
      if (rn <= hs->thr[r] || rn > 0.9 * rn_prev[r] || inner_cycles >= kMaxInner) {
        inner_done[r] = 1;
        continue;
      }
      rn_prev[r] = rn;
      hs->active[r] = 1;
      hs->beta0[r] = rn;
      ++n_active;
    }
    if (n_active == 0 || restarts >= P.max_restarts) {
      outer_next = true;  // the FP64 residual decides convergence (or the end)
      return LQCD_OK;
    }
  }
  LQCD_CUDA(cudaMemcpyAsync(B.st.active, hs->active, sizeof(int) * nrhs, cudaMemcpyHostToDevice, s), "up");
  LQCD_CUDA(cudaMemcpyAsync(B.st.thr, hs->thr, sizeof(double) * nrhs, cudaMemcpyHostToDevice, s), "up");
  LQCD_CUDA(cudaMemcpyAsync(d_beta0, hs->beta0, sizeof(double) * nrhs, cudaMemcpyHostToDevice, s), "up");
  *run = true;
  return LQCD_OK;
}

// One restart cycle on stream cs: v_0, m Arnoldi steps, back substitution, x += V y.
lqcd_status SolveJob::enqueue_cycle(cudaStream_t cs, bool allow_graph) {
  lqcd_status st;
  if (P.block) {
    int steps = 0;
    if ((st = block_gmres_cycle(ctx, P.op, nrhs, m, n_sys, B.basis, B.tmp_even_in, r64, sys_x, hs->thr,
                                hs->block_res, &hs->block_flag, &steps, cs)) != LQCD_OK)
      return st;
    for (int r = 0; r < nrhs; ++r)
      if (active_outer[r]) iters[r] += steps;
    // per step: operator, 2 x (Gram + reduction + update), 2 x (Gram + reduction + Cholesky + scale),
    // least-squares step; per cycle: v0, 2 x CholQR, ls init, solve, x update
    nl += (long long)steps * ((eo ? 2 : 1) + 6 + 8 + 1) + 1 + 8 + 1 + 2;
    ++restarts;
    return LQCD_OK;
  }
  LQCD_CUDA(launch_cycle_init(B.st, d_beta0, cs), "cycle init");
  LQCD_CUDA(launch_scale_convert(f64_inner, n_sys, nrhs, r64, B.st.scale, B.basis, cs, bf16), "v0");
  if (allow_graph) {
    if ((st = run_cycle(ctx, B, P.op, reorth, P.use_graph != 0, &prof, cs)) != LQCD_OK) return st;
  } else {
    if ((st = run_cycle_direct(ctx, B, P.op, reorth, &prof, cs)) != LQCD_OK) return st;
  }
  LQCD_CUDA(launch_backsub(B.st, cs), "backsub");
  if (B.ortho == 2) LQCD_CUDA(launch_dcgs_y(B.st, B.dc, cs), "dcgs y");
  LQCD_CUDA(launch_update_x(f64_inner, n_sys, nrhs, m, B.basis, n_sys, B.st.y, B.st.kmax, sys_x, cs, bf16),
            "update x");
  nl += cycle_launches();
  LQCD_CUDA(cudaMemcpyAsync(hs->kcycle, B.st.k, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, cs), "read k");
  pending_k = true;
  ++restarts;
  return LQCD_OK;
}

// Reconstruct x_e (odd-even), final full-operator residual, unpack and download x, stats.
lqcd_status SolveJob::finish() {
  lqcd_status st;
  if (x_cur != x64) {  // compacted: the last columns' solutions go back to the caller's block
    ColumnMap mp;
    for (int k = 0; k < nrhs; ++k) mp.col[k] = col[k];
    LQCD_CUDA(launch_repack_columns(ctx->g.V, layout_for(ctx, nrhs), layout_for(ctx, nrhs0), mp, true, x_cur, x64, s),
              "compaction scatter x");
    nl += 1;
  }
  for (int k = 0; k < nrhs; ++k) iters0[col[k]] += iters[k];
  // the rest runs on the caller's nrhs0 columns
  nrhs = nrhs0;
  n_full = (int64_t)packed_elems(ctx, LQCD_SITES_FULL, nrhs);
  n_half = n_full / 2;
  iters = iters0;
  bnorm = bnorm0;
  relres.assign(nrhs, 0.0);
  sys_x = eo ? (void*)((char*)x64 + (size_t)n_half * sizeof(double2)) : x64;
  if (eo && (st = schur_reconstruct(ctx, true, nrhs, b64, sys_x, x64, s)) != LQCD_OK) return st;
  if ((st = apply_operator(ctx, LQCD_OP_FULL, true, nrhs, x64, t64, nullptr, nullptr, s)) != LQCD_OK) return st;
  LQCD_CUDA(launch_sub_norm(plan_full, n_full, b64, t64, r64, red_partials, B.hn, s), "final residual");
  LQCD_CUDA(cudaMemcpyAsync(hs->rn2, B.hn, sizeof(double2) * nrhs, cudaMemcpyDeviceToHost, s), "read final");
  if (P.dagger)
    LQCD_CUDA(launch_gamma5_packed(n_full, nrhs, layout_for(ctx, nrhs).log_s, x64, s), "gamma5 x");
  if ((st = lqcd_unpack(ctx, LQCD_C128, LQCD_SITES_FULL, nrhs, x64, x_can, s)) != LQCD_OK) return st;
  if (x_host) LQCD_CUDA(cudaMemcpyAsync(x, x_can, full64, cudaMemcpyDeviceToHost, s), "download x");
  LQCD_CUDA(cudaStreamSynchronize(s), "final sync");
  nl += (eo ? 1 : 0) + 1 + 2 + 1;  // reconstruct, full operator, residual + reduction, unpack
  double relmax = 0.0;
  int itmax = 0;
  for (int r = 0; r < nrhs; ++r) {
    relres[r] = bnorm[r] > 0.0 ? std::sqrt(hs->rn2[2 * r]) / bnorm[r] : 0.0;
    relmax = std::max(relmax, relres[r]);
    itmax = std::max(itmax, iters[r]);
  }
  if (stats) {
    stats->status = result;
    stats->restarts = restarts;
    stats->iterations = itmax;
    stats->relres_max = relmax;
    stats->op_ms = prof.op_ms;
    stats->op_launches = prof.op_n;
    stats->op_bytes = prof.op_bytes;
    stats->ortho_ms = prof.gs_ms;
    stats->ortho_launches = prof.gs_n;
    stats->ortho_bytes = prof.gs_bytes;
    stats->kernel_launches = nl;
    stats->outer_steps = outer_steps;
    stats->ortho = B.ortho;
    if (stats->iters_per_rhs) for (int r = 0; r < nrhs; ++r) stats->iters_per_rhs[r] = iters[r];
    if (stats->relres_per_rhs) for (int r = 0; r < nrhs; ++r) stats->relres_per_rhs[r] = relres[r];
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (result == LQCD_NOT_CONVERGED)
    set_error(LQCD_NOT_CONVERGED, "lqcd_solve: max_restarts reached, max relative residual %.3e", relmax);
  return result;
}

}  // namespace lqcd

using namespace lqcd;


extern "C" {

lqcd_status lqcd_orthogonalise(lqcd_ctx ctx, lqcd_dtype dtype, lqcd_sites sites, int nrhs, int nvec,
                               const void* basis, void* w, void* h, void* hnorm, int reorth, void* stream) {
  if (!ctx) return set_error(LQCD_ERR_ARG, "lqcd_orthogonalise: null context");
  if ((dtype != LQCD_C64 && dtype != LQCD_C128 && dtype != LQCD_BF16S) || nrhs < 1 || nrhs > 256 || nvec < 1 ||
      nvec > 64 || !basis || !w || !h || !hnorm ||
      (sites != LQCD_SITES_FULL && sites != LQCD_SITES_EVEN && sites != LQCD_SITES_ODD) ||
      (dtype == LQCD_BF16S && nrhs > 32 && (nrhs % 2 != 0 || nrhs > 64)))
    return set_error(LQCD_ERR_ARG, "lqcd_orthogonalise: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const bool f64 = dtype == LQCD_C128;
  const bool bf16 = dtype == LQCD_BF16S;
  const int64_t n = (int64_t)packed_elems(ctx, sites, nrhs);
  BlasPlan plan = blas_plan(n, nrhs, ctx->num_sms);
  plan.wait_flag = wait_flag(ctx);
  void *partials, *h1, *h2, *hn;
  const size_t hb = sizeof(double2) * (size_t)(nvec + 1) * nrhs;
  lqcd_status st = workspace(ctx, "ortho_partials", hb * plan.blocks, &partials);
  if (st == LQCD_OK) st = workspace(ctx, "ortho_h1", hb, &h1);
  if (st == LQCD_OK) st = workspace(ctx, "ortho_h2", hb, &h2);
  if (st == LQCD_OK) st = workspace(ctx, "ortho_hn", hb, &hn);
  if (st != LQCD_OK) return st;
  LQCD_CUDA(launch_gs_pass(f64, plan, n, nvec, basis, n, w, nullptr, false, true, false, partials, h1, nullptr, s,
                           nullptr, bf16),
            "gs dots");
  if (reorth) {
    LQCD_CUDA(launch_gs_pass(f64, plan, n, nvec, basis, n, w, h1, true, true, false, partials, h2, nullptr, s,
                             nullptr, bf16),
              "gs update+dots");
    LQCD_CUDA(launch_gs_pass(f64, plan, n, nvec, basis, n, w, h2, true, false, true, partials, hn, nullptr, s,
                             nullptr, bf16),
              "gs update+norm");
  } else {
    LQCD_CUDA(launch_gs_pass(f64, plan, n, nvec, basis, n, w, h1, true, false, true, partials, hn, nullptr, s,
                             nullptr, bf16),
              "gs update+norm");
  }
  const int q = nvec * nrhs > nrhs ? nvec * nrhs : nrhs;
  combine_h_kernel<<<(q + 127) / 128, 128, 0, s>>>(nvec, nrhs, (const double2*)h1,
                                                   reorth ? (const double2*)h2 : nullptr, (const double2*)hn,
                                                   (double2*)h, (double*)hnorm);
  LQCD_CUDA(cudaGetLastError(), "combine h");
  return LQCD_OK;
}

lqcd_status lqcd_solve(lqcd_ctx ctx, const lqcd_solve_params* P, int nrhs, const void* b, void* x,
                       lqcd_solve_stats* stats, void* stream) {
  SolveJob job;
  cudaStream_t s = (cudaStream_t)stream;
  lqcd_status st = job.setup(ctx, P, nrhs, b, x, stats, s);
  if (st != LQCD_OK) return st;
  for (;;) {
    if ((st = job.enqueue_residual()) != LQCD_OK) return st;
    LQCD_CUDA(cudaStreamSynchronize(s), "sync residual");
    bool run = false;
    if ((st = job.decide(&run)) != LQCD_OK) return st;
    if (job.finished) break;
    if (!run) continue;   // the FP64 residual is due first
    if ((st = job.enqueue_cycle(s, true)) != LQCD_OK) return st;
  }
  return job.finish();
}

lqcd_status lqcd_solve_batch(int nlat, const lqcd_ctx* ctxs, const lqcd_solve_params* params, const int* nrhs,
                             const void* const* b, void* const* x, lqcd_solve_stats* stats, void* stream) {
  if (nlat < 1 || nlat > 64 || !ctxs || !params || !nrhs || !b || !x)
    return set_error(LQCD_ERR_ARG, "lqcd_solve_batch: bad arguments");
  for (int i = 0; i < nlat; ++i)
    for (int k = 0; k < i; ++k)
      if (ctxs[i] == ctxs[k]) return set_error(LQCD_ERR_ARG, "lqcd_solve_batch: lattice %d appears twice", i);
  for (int i = 0; i < nlat; ++i)
    if (params[i].block)
      return set_error(LQCD_ERR_ARG, "lqcd_solve_batch: block GMRES (params.block) is available in lqcd_solve only");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<SolveJob> jobs(nlat);
  lqcd_status st;
  for (int i = 0; i < nlat; ++i) {
    lqcd_solve_params pi = params[i];
    pi.profile = 0;   // CUDA events do not time kernels inside a graph
    if ((st = jobs[i].setup(ctxs[i], &pi, nrhs[i], b[i], x[i], stats ? &stats[i] : nullptr, s)) != LQCD_OK)
      return st;
  }
  // Per lattice a side stream; each restart round's cycles of every lattice still
  // running are captured once into one graph (fork/join over the side streams, so
  // the lattices' kernels run concurrently) and replayed as one launch per round.
  lqcd_ctx c0 = ctxs[0];
  if (!c0->capture_stream)
    LQCD_CUDA(cudaStreamCreateWithFlags(&c0->capture_stream, cudaStreamNonBlocking), "capture stream");
  std::vector<cudaStream_t> side(nlat, nullptr);
  std::vector<cudaEvent_t> ev(nlat + 1, nullptr);
  struct Cleanup {
    std::vector<cudaStream_t>* side;
    std::vector<cudaEvent_t>* ev;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    ~Cleanup() {
      if (ex) cudaGraphExecDestroy(ex);
      if (g) cudaGraphDestroy(g);
      for (auto h : *side) if (h) cudaStreamDestroy(h);
      for (auto e : *ev) if (e) cudaEventDestroy(e);
    }
  } cleanup{&side, &ev};
  for (int i = 0; i < nlat; ++i) LQCD_CUDA(cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking), "stream");
  for (auto& e : ev) LQCD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
  std::vector<char> running(nlat, 0);
  std::string graph_key;
  int rounds = 0;
  for (;;) {
    int n_run = 0;
    for (auto& j : jobs)
      if (!j.finished && (st = j.enqueue_residual()) != LQCD_OK) return st;
    LQCD_CUDA(cudaStreamSynchronize(s), "sync residuals");
    std::string key;
    for (int i = 0; i < nlat; ++i) {
      bool run = false;
      if (!jobs[i].finished && (st = jobs[i].decide(&run)) != LQCD_OK) return st;
      running[i] = run ? 1 : 0;
      n_run += run;
      key += run ? '1' : '0';
      key += std::to_string(jobs[i].compactions) + ',';   // a compacted lattice's branch is captured anew
    }
    bool all_finished = true;
    for (auto& j : jobs) all_finished = all_finished && j.finished;
    if (all_finished) break;
    if (n_run == 0) continue;   // only FP64 residuals are due this round
    if (key != graph_key) {   // the set of running lattices changed: capture the round anew
      if (cleanup.ex) { cudaGraphExecDestroy(cleanup.ex); cleanup.ex = nullptr; }
      if (cleanup.g) { cudaGraphDestroy(cleanup.g); cleanup.g = nullptr; }
      cudaStream_t cs = c0->capture_stream;
      LQCD_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "begin capture");
      lqcd_status cst = LQCD_OK;
      cudaError_t ce = cudaEventRecord(ev[nlat], cs);
      for (int i = 0; i < nlat && cst == LQCD_OK && ce == cudaSuccess; ++i) {
        if (!running[i]) continue;
        ce = cudaStreamWaitEvent(side[i], ev[nlat], 0);
        if (ce != cudaSuccess) break;
        const int restarts_before = jobs[i].restarts;
        cst = jobs[i].enqueue_cycle(side[i], false);
        jobs[i].restarts = restarts_before;   // restarts and launches are counted per replay below
        jobs[i].nl -= jobs[i].cycle_launches();
        if (cst != LQCD_OK) break;
        ce = cudaEventRecord(ev[i], side[i]);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(cs, ev[i], 0);
      }
      cudaGraph_t g = nullptr;
      cudaError_t ee = cudaStreamEndCapture(cs, &g);
      if (cst != LQCD_OK) { if (g) cudaGraphDestroy(g); return cst; }
      if (ce != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_error(ce, "batch capture"); }
      if (ee != cudaSuccess) return cuda_error(ee, "end capture");
      cleanup.g = g;
      LQCD_CUDA(cudaGraphInstantiate(&cleanup.ex, g, 0), "graph instantiate");
      graph_key = key;
    }
    LQCD_CUDA(cudaGraphLaunch(cleanup.ex, s), "graph launch");
    for (int i = 0; i < nlat; ++i)
      if (running[i]) {
        jobs[i].restarts += 1;
        jobs[i].pending_k = true;
        jobs[i].nl += jobs[i].cycle_launches();
      }
    ++rounds;
  }
  lqcd_status worst = LQCD_OK;
  for (auto& j : jobs) {
    st = j.finish();
    if (st < 0) return st;
    if (st != LQCD_OK) worst = st;
  }
  (void)rounds;
  return worst;
}

}  // extern "C"
