// Block GMRES: one block Krylov space for all rhs of a block (Sec. II's block Krylov
// solvers; the paper's Algorithm 2 instead runs the rhs in independent lockstep, see
// Sec. III-A-2). Used as the inner solver of the FP64 iterative refinement.
//
// For a block R0 of p right-hand sides (an n x p matrix: a packed block, whose rhs index
// is innermost, IS such a matrix with p contiguous entries per row), one cycle builds
//   R0 = V_0 S_0,  D V_j = sum_{i<=j} V_i H_ij + V_{j+1} H_{j+1,j}
// with p x p blocks H and orthonormal n x p blocks V_i: block classical Gram-Schmidt with
// one re-orthogonalisation (CGS2) against V_0..V_j, then the Cholesky QR of what is left,
// twice (CholQR2: G = W^H W = R^H R, W <- W R^{-1}). The block least-squares problem
// min_Y || E_1 S_0 - Hbar Y ||_F is kept in QR form: every new block column gets the
// Householder reflectors of the earlier columns and p new ones, which also update the
// rotated right-hand side G; the residual norm of rhs c after k steps is the norm of
// column c of G's last p rows. The cycle ends when every column's norm is below its
// threshold or after m steps; then Y solves R Y = G and x += V Y (FP64).
//
// Device work per step: the FP32 operator on V_j, four block passes of the CGS2
// (dots, update, dots, update; each dot pass a (j+1)p x p Gram reduction), two Gram +
// scale pairs of the CholQR2, and small FP64 kernels on one CTA (Cholesky, triangular
// inverses, the Householder step). The host reads the p residual norms after each step.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "ctx.h"

namespace lqcd {
namespace blk {

constexpr int kMaxP = 16;      // rhs per block
constexpr int kTileRows = 64;  // rows staged in shared memory per tile of the Gram kernel

// Partial block Gram matrices over this CTA's rows:
//   part[cta][i][a][b] = sum_rows conj(V_i[row][a]) W[row][b],  i < nblk
// V_i = V + i * vstride, rows of p complex numbers (stride p). Tiles of kTileRows rows of W
// and of V_i are staged in shared memory; thread (q, a, b) accumulates entry (a, b) of
// block i = i0 + q (256 / p^2 blocks per round).
__global__ void __launch_bounds__(256) gram_kernel(int64_t rows, int p, int nblk, const float2* __restrict__ V,
                                                   int64_t vstride, const float2* __restrict__ W,
                                                   double2* __restrict__ part) {
  __shared__ float2 ws[kTileRows * kMaxP];
  __shared__ float2 vs[kTileRows * kMaxP * 4];  // up to 4 blocks per round (p <= 8)
  const int pp = p * p;
  const int per_round = max(1, min(256 / pp, 4));
  const int q = threadIdx.x / pp, e = threadIdx.x % pp, a = e / p, b = e % p;
  const int64_t chunk = (rows + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = blockIdx.x * chunk, r1 = min(rows, r0 + chunk);
  for (int i0 = 0; i0 < nblk; i0 += per_round) {
    const int nb = min(per_round, nblk - i0);
    double2 acc = make_double2(0.0, 0.0);
    for (int64_t t = r0; t < r1; t += kTileRows) {
      const int tr = (int)min((int64_t)kTileRows, r1 - t);
      __syncthreads();
      for (int k = threadIdx.x; k < tr * p; k += blockDim.x) ws[k] = W[t * p + k];
      for (int k = threadIdx.x; k < nb * tr * p; k += blockDim.x) {
        const int bi = k / (tr * p), kk = k % (tr * p);
        vs[bi * kTileRows * p + kk] = V[(int64_t)(i0 + bi) * vstride + t * p + kk];
      }
      __syncthreads();
      if (q < nb) {
        float2 fa = make_float2(0.f, 0.f);
        const float2* vq = vs + q * kTileRows * p;
        for (int r = 0; r < tr; ++r) {
          const float2 v = vq[r * p + a], w = ws[r * p + b];
          fa.x += v.x * w.x + v.y * w.y;
          fa.y += v.x * w.y - v.y * w.x;
        }
        acc.x += fa.x;
        acc.y += fa.y;
      }
    }
    if (q < nb) part[((int64_t)blockIdx.x * nblk + i0 + q) * pp + e] = acc;
  }
}

// out[k] = sum over CTAs of part[cta][k] (fixed order), k < n.
__global__ void gram_reduce_kernel(int ctas, int n, const double2* __restrict__ part, double2* __restrict__ out) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    double2 s = make_double2(0.0, 0.0);
    for (int c = 0; c < ctas; ++c) {
      const double2 v = part[(int64_t)c * n + k];
      s.x += v.x;
      s.y += v.y;
    }
    out[k] = s;
  }
}

// Row-wise products with p x p matrices (coefficients staged in shared memory in FP32;
// lane b of a group of GS >= p lanes owns entry b of a row, shuffles broadcast the row):
//   MODE 0:  W[row] -= sum_{i < nblk} V_i[row] C_i            (C: [nblk][p][p], FP64)
//   MODE 1:  W[row]  = W[row] M                               (M: [p][p])
//   MODE 2:  X[row] += sum_{i < nblk} V_i[row] C_i, X FP64
template <int GS, int MODE>
__global__ void __launch_bounds__(256) rowmul_kernel(int64_t rows, int p, int nblk, const float2* __restrict__ V,
                                                     int64_t vstride, const double2* __restrict__ C, float2* W,
                                                     double2* X) {
  extern __shared__ float2 cs[];  // [nblk][p][p]
  for (int k = threadIdx.x; k < nblk * p * p; k += blockDim.x) cs[k] = make_float2((float)C[k].x, (float)C[k].y);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int b = lane % GS;
  const unsigned gmask = GS == 32 ? 0xffffffffu : (((1u << GS) - 1u) << (lane - b));
  const int64_t rows_per_cta = (int64_t)blockDim.x / GS;
  for (int64_t row = blockIdx.x * rows_per_cta + threadIdx.x / GS; row - (threadIdx.x / GS) < rows;
       row += (int64_t)gridDim.x * rows_per_cta) {
    const bool on = row < rows && b < p;
    if (MODE == 1) {
      const float2 w = on ? W[row * p + b] : make_float2(0.f, 0.f);
      float2 acc = make_float2(0.f, 0.f);
      for (int a = 0; a < p; ++a) {
        const float wx = __shfl_sync(gmask, w.x, a, GS), wy = __shfl_sync(gmask, w.y, a, GS);
        const float2 m = cs[a * p + (b < p ? b : 0)];
        acc.x += wx * m.x - wy * m.y;
        acc.y += wx * m.y + wy * m.x;
      }
      if (on) W[row * p + b] = acc;
    } else {
      float2 acc = make_float2(0.f, 0.f);
      for (int i = 0; i < nblk; ++i) {
        const float2 v = on ? V[(int64_t)i * vstride + row * p + b] : make_float2(0.f, 0.f);
        for (int a = 0; a < p; ++a) {
          const float vx = __shfl_sync(gmask, v.x, a, GS), vy = __shfl_sync(gmask, v.y, a, GS);
          const float2 c = cs[(i * p + a) * p + (b < p ? b : 0)];
          acc.x += vx * c.x - vy * c.y;
          acc.y += vx * c.y + vy * c.x;
        }
      }
      if (on) {
        if (MODE == 0) {
          const float2 w = W[row * p + b];
          W[row * p + b] = make_float2(w.x - acc.x, w.y - acc.y);
        } else {
          double2 x = X[row * p + b];
          x.x += acc.x;
          x.y += acc.y;
          X[row * p + b] = x;
        }
      }
    }
  }
}

// FP64 -> FP32 copy of a block.
__global__ void to_f32_kernel(int64_t n, const double2* __restrict__ a, float2* __restrict__ o) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    o[k] = make_float2((float)a[k].x, (float)a[k].y);
}

// ---------------------------------------------------------------- small dense FP64 state

struct Small {
  int p, m;
  double2* G;     // [p][p] Gram matrix of the block being normalised
  double2* R;     // [p][p] its Cholesky factor (upper), G = R^H R
  double2* Rinv;  // [p][p] R^{-1}
  double2* Racc;  // [p][p] product of the CholQR2 factors (S_0 or H_{j+1,j})
  double2* C1;    // [(m+1)][p][p] first Gram-Schmidt coefficients of the step
  double2* C2;    // [(m+1)][p][p] second ones
  double2* H;     // [m][(m+1)p][p] block columns, rotated in place to R of the least squares
  double2* hv;    // [m][p][2p] Householder vectors
  double* tau;    // [m][p] their factors
  double2* Gm;    // [(m+1)p][p] rotated right-hand side
  double2* Y;     // [m p][p] solution of the least squares
  double* res;    // [p] residual norm per rhs after the last step
  int* flag;      // 1: the Cholesky factorisation found a non-positive pivot
};

// Cholesky G = R^H R (upper R) and R^{-1}, one thread (p <= 16); mode 0: Racc = R,
// mode 1: Racc = R Racc. flag is set when a pivot is <= 1e-10 * max diag (rank deficiency).
__global__ void chol_kernel(Small s, int mode) {
  if (threadIdx.x != 0) return;
  const int p = s.p;
  double2 R[kMaxP * kMaxP], Ri[kMaxP * kMaxP];
  double dmax = 0.0;
  for (int i = 0; i < p; ++i) dmax = fmax(dmax, s.G[i * p + i].x);
  for (int i = 0; i < p * p; ++i) { R[i] = make_double2(0, 0); Ri[i] = make_double2(0, 0); }
  for (int j = 0; j < p; ++j) {
    // R[j][j] = sqrt(G[j][j] - sum_k |R[k][j]|^2); R[j][c] = (G[j][c] - sum_k conj(R[k][j]) R[k][c]) / R[j][j]
    double d = s.G[j * p + j].x;
    for (int k = 0; k < j; ++k) d -= R[k * p + j].x * R[k * p + j].x + R[k * p + j].y * R[k * p + j].y;
    // a pivot below 1e-10 of the largest diagonal entry: the block's columns are dependent to
    // within FP32 rounding (singular values below 1e-5 of the largest); its normalisation would
    // only amplify rounding noise
    if (!(d > 1e-10 * dmax)) {
      *s.flag = 1;
      d = fmax(d, 1e-10 * dmax + 1e-300);
    }
    const double rjj = sqrt(d);
    R[j * p + j] = make_double2(rjj, 0.0);
    for (int c = j + 1; c < p; ++c) {
      double2 v = s.G[j * p + c];
      for (int k = 0; k < j; ++k) {
        const double2 a = R[k * p + j], b = R[k * p + c];  // conj(a) * b
        v.x -= a.x * b.x + a.y * b.y;
        v.y -= a.x * b.y - a.y * b.x;
      }
      R[j * p + c] = make_double2(v.x / rjj, v.y / rjj);
    }
  }
  // upper triangular inverse by back substitution, column by column
  for (int c = 0; c < p; ++c) {
    for (int i = c; i >= 0; --i) {
      double2 v = make_double2(i == c ? 1.0 : 0.0, 0.0);
      for (int k = i + 1; k <= c; ++k) {
        const double2 a = R[i * p + k], b = Ri[k * p + c];
        v.x -= a.x * b.x - a.y * b.y;
        v.y -= a.x * b.y + a.y * b.x;
      }
      const double d = R[i * p + i].x;
      Ri[i * p + c] = make_double2(v.x / d, v.y / d);
    }
  }
  double2 acc[kMaxP * kMaxP];
  for (int i = 0; i < p; ++i)
    for (int c = 0; c < p; ++c) {
      double2 v = make_double2(0, 0);
      if (mode == 0) {
        v = R[i * p + c];
      } else {
        for (int k = 0; k < p; ++k) {
          const double2 a = R[i * p + k], b = s.Racc[k * p + c];
          v.x += a.x * b.x - a.y * b.y;
          v.y += a.x * b.y + a.y * b.x;
        }
      }
      acc[i * p + c] = v;
    }
  for (int i = 0; i < p * p; ++i) {
    s.R[i] = R[i];
    s.Rinv[i] = Ri[i];
    s.Racc[i] = acc[i];
  }
}

// Householder vector for x (length L): v = x + sign(x_0) ||x|| e_0, beta = -sign(x_0) ||x||,
// tau = 2 / (v^H v); (I - tau v v^H) x = beta e_0. Returns beta (x_0 replaced by v_0).
__device__ double2 householder(double2* x, int L, double* tau) {
  double nrm2 = 0.0;
  for (int r = 0; r < L; ++r) nrm2 += x[r].x * x[r].x + x[r].y * x[r].y;
  const double nrm = sqrt(nrm2);
  if (nrm == 0.0) {
    *tau = 0.0;
    return make_double2(0.0, 0.0);
  }
  const double a0 = hypot(x[0].x, x[0].y);
  const double2 ph = a0 > 0.0 ? make_double2(x[0].x / a0, x[0].y / a0) : make_double2(1.0, 0.0);
  // v_0 = x_0 + ph ||x||
  x[0] = make_double2(x[0].x + ph.x * nrm, x[0].y + ph.y * nrm);
  const double vv = nrm2 - a0 * a0 + (a0 + nrm) * (a0 + nrm);
  *tau = 2.0 / vv;
  return make_double2(-ph.x * nrm, -ph.y * nrm);
}

// y <- (I - tau v v^H) y over L entries.
__device__ __forceinline__ void apply_reflector(const double2* v, double tau, double2* y, int L, int ystride) {
  double2 d = make_double2(0, 0);
  for (int r = 0; r < L; ++r) {  // v^H y
    const double2 a = v[r], b = y[r * ystride];
    d.x += a.x * b.x + a.y * b.y;
    d.y += a.x * b.y - a.y * b.x;
  }
  d.x *= tau;
  d.y *= tau;
  for (int r = 0; r < L; ++r) {
    const double2 a = v[r];
    y[r * ystride].x -= a.x * d.x - a.y * d.y;
    y[r * ystride].y -= a.x * d.y + a.y * d.x;
  }
}

// Block column j of the least squares: H[j] holds [C1 + C2 for blocks 0..j ; Racc = H_{j+1,j}]
// ((j+2)p x p, column c of row r at r * p + c). Apply the reflectors of columns 0..j-1, then p
// new ones on rows [jp, jp + 2p), which also rotate Gm; res[c] = ||Gm[(j+1)p.., c]||.
// One CTA; thread c < p owns column c (the reflector applications are column-independent).
__global__ void ls_step_kernel(Small s, int j) {
  const int p = s.p;
  const int c = threadIdx.x;
  double2* h = s.H + (int64_t)j * (s.m + 1) * p * p;  // [(m+1)p][p]
  if (c < p) {
    // assemble the column: blocks 0..j from C1 + C2, block j+1 from Racc (upper triangular)
    for (int i = 0; i <= j; ++i)
      for (int a = 0; a < p; ++a) {
        const double2 u = s.C1[(i * p + a) * p + c], w = s.C2[(i * p + a) * p + c];
        h[(i * p + a) * p + c] = make_double2(u.x + w.x, u.y + w.y);
      }
    for (int a = 0; a < p; ++a) h[((j + 1) * p + a) * p + c] = s.Racc[a * p + c];
    // earlier reflectors
    for (int k = 0; k < j; ++k)
      for (int i = 0; i < p; ++i) {
        const int L = 2 * p - i;
        apply_reflector(s.hv + ((int64_t)k * p + i) * 2 * p, s.tau[k * p + i], h + (k * p + i) * p + c, L, p);
      }
  }
  __syncthreads();
  // new reflectors: column i of the 2p x p block at rows jp + i .. jp + 2p - 1
  __shared__ double2 beta_s;
  for (int i = 0; i < p; ++i) {
    double2* vi = s.hv + ((int64_t)j * p + i) * 2 * p;
    const int L = 2 * p - i;
    if (c == 0) {
      for (int r = 0; r < L; ++r) vi[r] = h[(j * p + i + r) * p + i];
      double t;
      beta_s = householder(vi, L, &t);
      s.tau[j * p + i] = t;
    }
    __syncthreads();
    if (c < p && c > i)
      apply_reflector(vi, s.tau[j * p + i], h + (j * p + i) * p + c, L, p);
    if (c < p)  // rotated right-hand side
      apply_reflector(vi, s.tau[j * p + i], s.Gm + (j * p + i) * p + c, L, p);
    __syncthreads();
    if (c == 0) {
      h[(j * p + i) * p + i] = beta_s;
      for (int r = 1; r < L; ++r) h[(j * p + i + r) * p + i] = make_double2(0, 0);
    }
    __syncthreads();
  }
  if (c < p) {
    double n2 = 0.0;
    for (int a = 0; a < p; ++a) {
      const double2 g = s.Gm[((j + 1) * p + a) * p + c];
      n2 += g.x * g.x + g.y * g.y;
    }
    s.res[c] = sqrt(n2);
  }
}

// Gm = [S_0 (= Racc); 0], the least-squares right-hand side of a new cycle.
__global__ void ls_init_kernel(Small s) {
  const int p = s.p;
  for (int k = threadIdx.x; k < (s.m + 1) * p * p; k += blockDim.x)
    s.Gm[k] = k < p * p ? s.Racc[k] : make_double2(0, 0);
  if (threadIdx.x == 0) *s.flag = 0;
}

// Y = R^{-1} Gm[0 : kp] by back substitution on the rotated block columns 0..k-1 (R's
// column block i is H[i] rows 0..(i+1)p). One thread per rhs column.
__global__ void ls_solve_kernel(Small s, int k) {
  const int p = s.p;
  const int c = threadIdx.x;
  if (c >= p) return;
  const int n = k * p;
  for (int r = n - 1; r >= 0; --r) {
    double2 v = s.Gm[r * p + c];
    for (int q = r + 1; q < n; ++q) {
      const double2* hq = s.H + (int64_t)(q / p) * (s.m + 1) * p * p;
      const double2 a = hq[r * p + (q % p)], y = s.Y[q * p + c];
      v.x -= a.x * y.x - a.y * y.y;
      v.y -= a.x * y.y + a.y * y.x;
    }
    const double2* hr = s.H + (int64_t)(r / p) * (s.m + 1) * p * p;
    const double2 d = hr[r * p + (r % p)];
    const double dd = d.x * d.x + d.y * d.y;
    s.Y[r * p + c] = dd > 0.0 ? make_double2((v.x * d.x + v.y * d.y) / dd, (v.y * d.x - v.x * d.y) / dd)
                              : make_double2(0, 0);
  }
}

}  // namespace blk

// ---------------------------------------------------------------- host side

struct BlockGmres {
  lqcd_ctx ctx;
  int p, m;
  int64_t rows;      // n_sys / p
  int grid;          // CTAs of the Gram kernel
  void* basis;       // (m+1) FP32 blocks, stride n_sys
  int64_t n_sys;
  void* part;        // Gram partials [grid][m+1][p][p]
  blk::Small s;

  cudaError_t gram(int nblk, const void* V, const void* W, double2* out, cudaStream_t st) {
    blk::gram_kernel<<<grid, 256, 0, st>>>(rows, p, nblk, (const float2*)V, n_sys, (const float2*)W, (double2*)part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int n = nblk * p * p;
    blk::gram_reduce_kernel<<<(n + 255) / 256, 256, 0, st>>>(grid, n, (const double2*)part, out);
    return cudaGetLastError();
  }
  template <int MODE>
  cudaError_t rowmul_gs(int nblk, const void* V, const double2* C, void* W, void* X, cudaStream_t st) {
    const size_t smem = sizeof(float2) * (size_t)nblk * p * p;
    const int gs = p <= 1 ? 1 : p <= 2 ? 2 : p <= 4 ? 4 : p <= 8 ? 8 : 16;
    const int64_t rows_per_cta = 256 / gs;
    int64_t ctas = (rows + rows_per_cta - 1) / rows_per_cta;
    if (ctas > (int64_t)ctx->num_sms * 8) ctas = (int64_t)ctx->num_sms * 8;
    // coefficients of up to 65 blocks of 16 x 16: beyond the default 48 KB of dynamic shared memory
#define LQCD_RM(G)                                                                                              \
  {                                                                                                             \
    static std::once_flag attr;                                                                                 \
    std::call_once(attr, [] {                                                                                   \
      cudaFuncSetAttribute(blk::rowmul_kernel<G, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,            \
                           (int)(sizeof(float2) * 65 * blk::kMaxP * blk::kMaxP));                               \
    });                                                                                                         \
    blk::rowmul_kernel<G, MODE><<<(int)ctas, 256, smem, st>>>(rows, p, nblk, (const float2*)V, n_sys, C,        \
                                                              (float2*)W, (double2*)X);                         \
  }
    switch (gs) {
      case 1: LQCD_RM(1); break;
      case 2: LQCD_RM(2); break;
      case 4: LQCD_RM(4); break;
      case 8: LQCD_RM(8); break;
      default: LQCD_RM(16); break;
    }
#undef LQCD_RM
    return cudaGetLastError();
  }
  // W <- W R^{-1} twice (CholQR2); Racc = R2 R1. cholesky flag in s.flag.
  cudaError_t cholqr2(void* W, cudaStream_t st) {
    for (int pass = 0; pass < 2; ++pass) {
      cudaError_t e = gram(1, W, W, s.G, st);
      if (e != cudaSuccess) return e;
      blk::chol_kernel<<<1, 32, 0, st>>>(s, pass);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if ((e = rowmul_gs<1>(1, nullptr, s.Rinv, W, nullptr, st)) != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
};

// One block GMRES(m) cycle on the correction equation D e = r for the job's current
// columns: r is the FP64 residual r64 (n_sys elements), x (FP64) += e. thr[c]: the
// residual norm at which column c is done. h_res (p doubles) and h_flag: pinned host
// memory for the per-step residual norms and the rank-deficiency flag. Synchronises the
// stream after each step. Returns the number of steps taken in *steps.
lqcd_status block_gmres_cycle(lqcd_ctx ctx, int op, int nrhs, int m, int64_t n_sys, void* basis, void* tmp_even,
                              const void* r64, void* x64, const double* thr, double* h_res, int* h_flag, int* steps,
                              cudaStream_t st) {
  if (nrhs > blk::kMaxP) return set_error(LQCD_ERR_ARG, "block GMRES: at most %d rhs per block", blk::kMaxP);
  BlockGmres bg;
  bg.ctx = ctx;
  bg.p = nrhs;
  bg.m = m;
  bg.n_sys = n_sys;
  bg.rows = n_sys / nrhs;
  bg.basis = basis;
  bg.grid = std::max(1, std::min(2 * ctx->num_sms, (int)((bg.rows + blk::kTileRows - 1) / blk::kTileRows)));
  const int p = nrhs, pp = nrhs * nrhs;
  lqcd_status rs;
  if ((rs = workspace(ctx, "block_partials", sizeof(double2) * (size_t)bg.grid * (m + 1) * pp, &bg.part)) != LQCD_OK)
    return rs;
  const size_t sz[13] = {sizeof(double2) * pp, sizeof(double2) * pp, sizeof(double2) * pp, sizeof(double2) * pp,
                         sizeof(double2) * (size_t)(m + 1) * pp, sizeof(double2) * (size_t)(m + 1) * pp,
                         sizeof(double2) * (size_t)m * (m + 1) * pp, sizeof(double2) * (size_t)m * p * 2 * p,
                         sizeof(double) * (size_t)m * p, sizeof(double2) * (size_t)(m + 1) * pp,
                         sizeof(double2) * (size_t)m * pp, sizeof(double) * p, sizeof(int)};
  size_t total = 0;
  for (size_t q : sz) total += (q + 255) & ~(size_t)255;
  void* mem;
  if ((rs = workspace(ctx, "block_small", total, &mem)) != LQCD_OK) return rs;
  {
    char* q = (char*)mem;
    int k = 0;
    auto take = [&]() { void* r = q; q += (sz[k++] + 255) & ~(size_t)255; return r; };
    bg.s.p = p;
    bg.s.m = m;
    bg.s.G = (double2*)take();
    bg.s.R = (double2*)take();
    bg.s.Rinv = (double2*)take();
    bg.s.Racc = (double2*)take();
    bg.s.C1 = (double2*)take();
    bg.s.C2 = (double2*)take();
    bg.s.H = (double2*)take();
    bg.s.hv = (double2*)take();
    bg.s.tau = (double*)take();
    bg.s.Gm = (double2*)take();
    bg.s.Y = (double2*)take();
    bg.s.res = (double*)take();
    bg.s.flag = (int*)take();
  }
  const size_t vbytes = (size_t)n_sys * sizeof(float2);
  char* base = (char*)basis;
  // V_0 = R0 R^{-1}, S_0 = R
  blk::to_f32_kernel<<<std::min<int64_t>((n_sys + 255) / 256, 65535LL * 8), 256, 0, st>>>(n_sys, (const double2*)r64,
                                                                                        (float2*)base);
  LQCD_CUDA(cudaGetLastError(), "block v0");
  LQCD_CUDA(cudaMemsetAsync(bg.s.flag, 0, sizeof(int), st), "block flag");
  LQCD_CUDA(bg.cholqr2(base, st), "block QR of R0");
  blk::ls_init_kernel<<<1, 256, 0, st>>>(bg.s);
  LQCD_CUDA(cudaGetLastError(), "block ls init");
  int k = 0;
  for (int j = 0; j < m; ++j) {
    void* vj = base + (size_t)j * vbytes;
    void* w = base + (size_t)(j + 1) * vbytes;
    if ((rs = apply_operator(ctx, op, false, nrhs, vj, w, tmp_even, nullptr, st)) != LQCD_OK) return rs;
    // block CGS2 against V_0..V_j
    LQCD_CUDA(bg.gram(j + 1, base, w, bg.s.C1, st), "block dots 1");
    LQCD_CUDA(bg.rowmul_gs<0>(j + 1, base, bg.s.C1, w, nullptr, st), "block update 1");
    LQCD_CUDA(bg.gram(j + 1, base, w, bg.s.C2, st), "block dots 2");
    LQCD_CUDA(bg.rowmul_gs<0>(j + 1, base, bg.s.C2, w, nullptr, st), "block update 2");
    LQCD_CUDA(bg.cholqr2(w, st), "block QR");
    blk::ls_step_kernel<<<1, 32, 0, st>>>(bg.s, j);
    LQCD_CUDA(cudaGetLastError(), "block ls step");
    LQCD_CUDA(cudaMemcpyAsync(h_res, bg.s.res, sizeof(double) * p, cudaMemcpyDeviceToHost, st), "read res");
    LQCD_CUDA(cudaMemcpyAsync(h_flag, bg.s.flag, sizeof(int), cudaMemcpyDeviceToHost, st), "read flag");
    LQCD_CUDA(cudaStreamSynchronize(st), "block step sync");
    bool finite = true, done = true;
    for (int c = 0; c < p; ++c) {
      finite = finite && std::isfinite(h_res[c]);
      done = done && h_res[c] <= thr[c];
    }
    // A non-finite estimate: step j is discarded (its reflectors act on rows >= j p only, so the
    // least squares of steps 0..j-1 stand). A rank-deficient new block (the block form of a happy
    // breakdown, or FP32 rounding in a nearly dependent block): step j is kept, the cycle ends.
    if (!finite) break;
    k = j + 1;
    if (done || *h_flag) break;
  }
  blk::ls_solve_kernel<<<1, 32, 0, st>>>(bg.s, k);
  LQCD_CUDA(cudaGetLastError(), "block ls solve");
  LQCD_CUDA(bg.rowmul_gs<2>(k, base, bg.s.Y, nullptr, x64, st), "block update x");
  *steps = k;
  return LQCD_OK;
}

}  // namespace lqcd
