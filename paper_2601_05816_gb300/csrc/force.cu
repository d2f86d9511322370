// Gradient of L = sum_i Re <eta_i, x_i>, x_i = D^{-1} b_i, with respect to the gauge links
// (the differentiable solve; the paper has no adjoint).
//
// With lambda_i = D^{-dagger} eta_i (the adjoint solve), dL = -Re <lambda, (dD) x>. The
// gradient G (PyTorch's convention for a real loss: dL = Re sum conj(G) dU over the link
// entries) has two parts:
//
// * hopping terms of D (Sec. III-A-1): D x holds -pi^-_mu b U_mu(y) x(y+mu) at y and
//   -pi^+_mu (b U_mu(y))^dag x(y) at y+mu (b: the time boundary factor of the link), so
//     G_mu(y) += b [conj(M) + N^T],  M_ab = sum_s conj(lam_sa(y)) (pi^- x(y+mu))_sb,
//                                    N_ab = sum_s conj(lam_sa(y+mu)) (pi^+ x(y))_sb
//   (outer products of the projected spinors, summed over rhs): force_hop_kernel.
// * clover term C(x) = (c_sw/32) sum_{mu != nu} gamma_mu gamma_nu (x) (Q_mu,nu - Q_nu,mu),
//   D = ... - C: dL = Re sum_x lam^H dC x. With W_mu,nu = (c_sw/32) sum_{i,s}
//   (gamma_mu gamma_nu x_i)_s lam_i,s^H, Q_nu,mu = Q_mu,nu^dag and W_nu,mu = -W_mu,nu this is
//     dL = Re sum_x sum_{mu<nu} tr[dQ_mu,nu(x) Y(x)],  Y = 2 (W_mu,nu - W_mu,nu^dag).
//   For a leaf A F B of Q_mu,nu(x) the factor F = U_rho(y) (or U_rho(y)^dag) gets
//   K = B Y A: G_rho(y) += K^dag (or K). force_leaf_kernel writes K for every
//   (site, plane, leaf, factor) into a buffer, force_gather_kernel sums, per link, its
//   24 entries in a fixed order (deterministic).
//
// The links come from the packed FP64 copy, whose time links on t = T-1 carry the
// boundary factor b. In a clover leaf the other factors then contain b exactly once when
// the differentiated link is such a time link (the plaquette's two time links lie on the
// same time slice) and b^2 = 1 otherwise; the hopping part also carries b on those links.
// So the gather multiplies the sum of both parts by b on the time links of t = T-1.
//
// Layouts: x, lambda canonical complex128 [nrhs][V][4][3]; G canonical complex128
// [V][4][3][3] (site number with the last coordinate fastest, like the gauge input).
#include "ctx.h"

namespace lqcd {
namespace {

struct M3 {
  double2 e[9];
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ M3 mm(const M3& a, const M3& b) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double2 s = make_double2(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double2 p = cmul(a.e[3 * i + k], b.e[3 * k + j]);
        s.x += p.x;
        s.y += p.y;
      }
      c.e[3 * i + j] = s;
    }
  return c;
}
__device__ __forceinline__ M3 dag(const M3& a) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) c.e[3 * i + j] = make_double2(a.e[3 * j + i].x, -a.e[3 * j + i].y);
  return c;
}
__device__ __forceinline__ M3 eye3() {
  M3 c;
#pragma unroll
  for (int i = 0; i < 9; ++i) c.e[i] = make_double2((i % 4 == 0) ? 1.0 : 0.0, 0.0);
  return c;
}

// gamma_mu in the chiral basis, gamma = [[0, P], [P^dag, 0]] with P_t = 1, P_z = i sigma_z,
// P_y = i sigma_y, P_x = i sigma_x (mu = 0, 1, 2, 3 is t, z, y, x): row-major 2x2 P per mu.
__constant__ double2 kP[4][4] = {
    {{1, 0}, {0, 0}, {0, 0}, {1, 0}},
    {{0, 1}, {0, 0}, {0, 0}, {0, -1}},
    {{0, 0}, {1, 0}, {-1, 0}, {0, 0}},
    {{0, 0}, {0, 1}, {0, 1}, {0, 0}},
};

// out = gamma_mu in (4 spins x 3 colours): upper = P lower, lower = P^dag upper.
__device__ __forceinline__ void gamma_apply(int mu, const double2 (&in)[4][3], double2 (&out)[4][3]) {
  const double2 p00 = kP[mu][0], p01 = kP[mu][1], p10 = kP[mu][2], p11 = kP[mu][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double2 u0 = cmul(p00, in[2][a]), u1 = cmul(p01, in[3][a]);
    const double2 u2 = cmul(p10, in[2][a]), u3 = cmul(p11, in[3][a]);
    out[0][a] = make_double2(u0.x + u1.x, u0.y + u1.y);
    out[1][a] = make_double2(u2.x + u3.x, u2.y + u3.y);
    // P^dag: (P^dag)_ij = conj(P_ji)
    const double2 d0 = cmulc(p00, in[0][a]), d1 = cmulc(p10, in[1][a]);
    const double2 d2 = cmulc(p01, in[0][a]), d3 = cmulc(p11, in[1][a]);
    out[2][a] = make_double2(d0.x + d1.x, d0.y + d1.y);
    out[3][a] = make_double2(d2.x + d3.x, d2.y + d3.y);
  }
}

__device__ __forceinline__ void load_spinor(const double2* p, double2 (&s)[4][3]) {
#pragma unroll
  for (int k = 0; k < 12; ++k) s[k / 3][k % 3] = p[k];
}

// coordinates of a site number (last coordinate fastest)
__device__ __forceinline__ void lex_coords(const Geom& g, int lex, int (&c)[4]) {
  c[3] = lex % g.X;
  int r = lex / g.X;
  c[2] = r % g.Y;
  r /= g.Y;
  c[1] = r % g.Z;
  c[0] = r / g.Z;
}
__device__ __forceinline__ int coords_lex(const Geom& g, const int (&c)[4]) {
  return ((c[0] * g.Z + c[1]) * g.Y + c[2]) * g.X + c[3];
}
__device__ __forceinline__ int extent(const Geom& g, int mu) {
  return mu == 0 ? g.T : (mu == 1 ? g.Z : (mu == 2 ? g.Y : g.X));
}
__device__ __forceinline__ int eo_index(const Geom& g, int lex, const int (&c)[4]) {
  return ((c[0] + c[1] + c[2] + c[3]) & 1) * g.Vh + (lex >> 1);
}

// Hopping part, one thread per (site y, direction mu): G_mu(y) = conj(M) + N^T (without the
// boundary factor, applied by the gather).
__global__ void __launch_bounds__(128) force_hop_kernel(Geom g, int nrhs, const double2* __restrict__ x,
                                                        const double2* __restrict__ lam, double2* __restrict__ G) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 4 * g.V) return;
  const int y = idx >> 2, mu = idx & 3;
  int c[4];
  lex_coords(g, y, c);
  c[mu] = (c[mu] + 1) % extent(g, mu);
  const int yf = coords_lex(g, c);
  double2 M[9], N[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) { M[i] = make_double2(0.0, 0.0); N[i] = make_double2(0.0, 0.0); }
  for (int n = 0; n < nrhs; ++n) {
    const int64_t base = (int64_t)n * g.V;
    double2 xf[4][3], xh[4][3], gf[4][3], gh[4][3], ly[4][3], lf[4][3];
    load_spinor(x + (base + yf) * 12, xf);
    load_spinor(x + (base + y) * 12, xh);
    load_spinor(lam + (base + y) * 12, ly);
    load_spinor(lam + (base + yf) * 12, lf);
    gamma_apply(mu, xf, gf);
    gamma_apply(mu, xh, gh);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const double2 pm = make_double2(0.5 * (xf[s][b].x - gf[s][b].x), 0.5 * (xf[s][b].y - gf[s][b].y));
        const double2 pp = make_double2(0.5 * (xh[s][b].x + gh[s][b].x), 0.5 * (xh[s][b].y + gh[s][b].y));
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const double2 m = cmulc(ly[s][a], pm), q = cmulc(lf[s][a], pp);
          M[3 * a + b].x += m.x; M[3 * a + b].y += m.y;
          N[3 * a + b].x += q.x; N[3 * a + b].y += q.y;
        }
      }
  }
  double2* out = G + (int64_t)idx * 9;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      out[3 * a + b] = make_double2(M[3 * a + b].x + N[3 * b + a].x, -M[3 * a + b].y + N[3 * b + a].y);
}

// The six planes (mu < nu) and the four leaves of Q_mu,nu(x): factor q of leaf k is the link
// in direction (0: mu, 1: nu) at x + dmu mu-hat + dnu nu-hat, daggered or not.
__constant__ int kPlane[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
struct LeafFactor {
  signed char dir, dmu, dnu, dag;
};
__constant__ LeafFactor kLeaf[4][4] = {
    {{0, 0, 0, 0}, {1, 1, 0, 0}, {0, 0, 1, 1}, {1, 0, 0, 1}},
    {{1, 0, 0, 0}, {0, -1, 1, 1}, {1, -1, 0, 1}, {0, -1, 0, 0}},
    {{0, -1, 0, 1}, {1, -1, -1, 1}, {0, -1, -1, 0}, {1, 0, -1, 0}},
    {{1, 0, -1, 1}, {0, 0, -1, 0}, {1, 1, -1, 0}, {0, 0, 0, 1}},
};

__device__ __forceinline__ M3 load_link(const Geom& g, const double2* links, int lex, const int (&c)[4], int rho) {
  const int e = eo_index(g, lex, c);
  M3 u;
#pragma unroll
  for (int k = 0; k < 9; ++k) u.e[k] = links[(int64_t)(rho * 9 + k) * g.V + e];
  return u;
}

// Clover part, one thread per (site x, plane): Y = 2 (W - W^dag), then K = B Y A for every
// factor of every leaf, written to buf[((x * 6 + plane) * 4 + leaf) * 4 + factor][9].
__global__ void __launch_bounds__(128) force_leaf_kernel(Geom g, int nrhs, double cfac, const double2* __restrict__ x,
                                                         const double2* __restrict__ lam,
                                                         const double2* __restrict__ links, double2* __restrict__ buf) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 6 * g.V) return;
  const int xs = idx / 6, pl = idx % 6;
  const int mu = kPlane[pl][0], nu = kPlane[pl][1];
  // W = cfac * sum_{i,s} (gamma_mu gamma_nu x_i)_s lam_i,s^H, W_ba
  M3 W;
#pragma unroll
  for (int i = 0; i < 9; ++i) W.e[i] = make_double2(0.0, 0.0);
  for (int n = 0; n < nrhs; ++n) {
    const int64_t base = ((int64_t)n * g.V + xs) * 12;
    double2 xv[4][3], t[4][3], gg[4][3], lv[4][3];
    load_spinor(x + base, xv);
    load_spinor(lam + base, lv);
    gamma_apply(nu, xv, t);
    gamma_apply(mu, t, gg);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const double2 p = cmulc(lv[s][a], gg[s][b]);
          W.e[3 * b + a].x += p.x;
          W.e[3 * b + a].y += p.y;
        }
  }
  M3 Y;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double2 w = W.e[3 * i + j], wt = W.e[3 * j + i];
      Y.e[3 * i + j] = make_double2(2.0 * cfac * (w.x - wt.x), 2.0 * cfac * (w.y + wt.y));
    }
  int c0[4];
  lex_coords(g, xs, c0);
  const int ext_mu = extent(g, mu), ext_nu = extent(g, nu);
  for (int k = 0; k < 4; ++k) {
    M3 F[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const LeafFactor f = kLeaf[k][q];
      int c[4] = {c0[0], c0[1], c0[2], c0[3]};
      c[mu] = (c[mu] + f.dmu + ext_mu) % ext_mu;
      c[nu] = (c[nu] + f.dnu + ext_nu) % ext_nu;
      const M3 u = load_link(g, links, coords_lex(g, c), c, f.dir == 0 ? mu : nu);
      F[q] = f.dag ? dag(u) : u;
    }
    // suffix products B_q = F_{q+1} ... F_3
    M3 Bs[4];
    Bs[3] = eye3();
    Bs[2] = F[3];
    Bs[1] = mm(F[2], F[3]);
    Bs[0] = mm(F[1], Bs[1]);
    M3 A = eye3();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const M3 K = mm(mm(Bs[q], Y), A);
      double2* out = buf + ((((int64_t)xs * 6 + pl) * 4 + k) * 4 + q) * 9;
#pragma unroll
      for (int i = 0; i < 9; ++i) out[i] = K.e[i];
      if (q < 3) A = (q == 0) ? F[0] : mm(A, F[q]);
    }
  }
}

// Per link (site y, direction rho): the 24 leaf contributions in a fixed order, added to the
// hopping part; then the boundary factor on the time links of t = T-1.
__global__ void __launch_bounds__(128) force_gather_kernel(Geom g, int time_bc, int clover,
                                                           const double2* __restrict__ buf,
                                                           double2* __restrict__ G) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 4 * g.V) return;
  const int y = idx >> 2, rho = idx & 3;
  int cy[4];
  lex_coords(g, y, cy);
  double2 acc[9];
  double2* out = G + (int64_t)idx * 9;
#pragma unroll
  for (int i = 0; i < 9; ++i) acc[i] = out[i];
  if (clover) {
    for (int pl = 0; pl < 6; ++pl) {
      const int mu = kPlane[pl][0], nu = kPlane[pl][1];
      if (mu != rho && nu != rho) continue;
      const int dir = (rho == mu) ? 0 : 1;
      const int ext_mu = extent(g, mu), ext_nu = extent(g, nu);
      for (int k = 0; k < 4; ++k)
        for (int q = 0; q < 4; ++q) {
          const LeafFactor f = kLeaf[k][q];
          if (f.dir != dir) continue;
          // the leaf starts at x = y - offset
          int c[4] = {cy[0], cy[1], cy[2], cy[3]};
          c[mu] = (c[mu] - f.dmu + ext_mu) % ext_mu;
          c[nu] = (c[nu] - f.dnu + ext_nu) % ext_nu;
          const double2* K = buf + ((((int64_t)coords_lex(g, c) * 6 + pl) * 4 + k) * 4 + q) * 9;
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
              // daggered factor: G += K; plain factor: G += K^dag
              const double2 v = f.dag ? K[3 * i + j] : make_double2(K[3 * j + i].x, -K[3 * j + i].y);
              acc[3 * i + j].x += v.x;
              acc[3 * i + j].y += v.y;
            }
        }
    }
  }
  const double b = (rho == 0 && cy[0] == g.T - 1) ? (double)time_bc : 1.0;
#pragma unroll
  for (int i = 0; i < 9; ++i) out[i] = make_double2(b * acc[i].x, b * acc[i].y);
}

// gamma5 = diag(-1, -1, 1, 1) on a packed block: negate the components of spins 0 and 1.
__global__ void gamma5_packed_kernel(int64_t n, int nrhs, int log_s, double2* __restrict__ v) {
  const int64_t run = ((int64_t)1 << log_s) * nrhs;  // elements per component run
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int comp = (int)((e / run) % 12);
    if (comp < 6) v[e] = make_double2(-v[e].x, -v[e].y);
  }
}

}  // namespace

cudaError_t launch_gamma5_packed(int64_t n, int nrhs, int log_s, void* v, cudaStream_t s) {
  const int threads = 256;
  int64_t blocks = (n + threads - 1) / threads;
  if (blocks > 65535 * 16) blocks = 65535 * 16;
  gamma5_packed_kernel<<<(int)blocks, threads, 0, s>>>(n, nrhs, log_s, (double2*)v);
  return cudaGetLastError();
}

}  // namespace lqcd

using namespace lqcd;

extern "C" lqcd_status lqcd_force(lqcd_ctx ctx, int nrhs, const void* x, const void* lambda, void* grad_U,
                                  void* stream) {
  if (!ctx) return set_error(LQCD_ERR_ARG, "lqcd_force: null context");
  if (!x || !lambda || !grad_U || nrhs < 1 || nrhs > 256)
    return set_error(LQCD_ERR_ARG, "lqcd_force: bad arguments");
  if (!ctx->have_gauge || !ctx->have_blocks)
    return set_error(LQCD_ERR_STATE, "lqcd_force: set_gauge and set_clover must be called first");
  if (!is_device_pointer(x) || !is_device_pointer(lambda) || !is_device_pointer(grad_U))
    return set_error(LQCD_ERR_ARG, "lqcd_force: x, lambda and grad_U must be device pointers");
  cudaStream_t s = (cudaStream_t)stream;
  const Geom& g = ctx->g;
  const int threads = 128;
  force_hop_kernel<<<(4 * g.V + threads - 1) / threads, threads, 0, s>>>(g, nrhs, (const double2*)x,
                                                                        (const double2*)lambda, (double2*)grad_U);
  LQCD_CUDA(cudaGetLastError(), "force hop");
  const bool clover = ctx->c_sw != 0.0;
  void* buf = nullptr;
  if (clover) {
    lqcd_status st = workspace(ctx, "force_leaves", (size_t)g.V * 6 * 16 * 9 * sizeof(double2), &buf);
    if (st != LQCD_OK) return st;
    force_leaf_kernel<<<(6 * g.V + threads - 1) / threads, threads, 0, s>>>(
        g, nrhs, ctx->c_sw / 32.0, (const double2*)x, (const double2*)lambda, (const double2*)ctx->links64,
        (double2*)buf);
    LQCD_CUDA(cudaGetLastError(), "force leaves");
  }
  force_gather_kernel<<<(4 * g.V + threads - 1) / threads, threads, 0, s>>>(g, ctx->time_bc, clover ? 1 : 0,
                                                                           (const double2*)buf,
                                                                           (double2*)grad_U);
  LQCD_CUDA(cudaGetLastError(), "force gather");
  return LQCD_OK;
}
