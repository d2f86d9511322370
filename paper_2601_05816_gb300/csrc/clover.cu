// Clover term and site blocks (Sec. III-A-1: D = D_W - C, C Hermitian block-diagonal
// with 42 complex numbers per site; Sec. III-A-2: A_ee^{-1} of the Schur complement).
//
//   C(x) = (c_sw/32) sum_{mu != nu} gamma_mu gamma_nu (x) (Q_mu,nu(x) - Q_nu,mu(x)),
// Q_mu,nu the clover-leaf sum of the four plaquettes in the (mu, nu) plane that
// start and end at x. Because Q_nu,mu = Q_mu,nu^dag and gamma_nu gamma_mu =
// -gamma_mu gamma_nu, the sum is (c_sw/16) sum_{mu<nu} gamma_mu gamma_nu (x) F_mu,nu with
// F = Q - Q^dag. In the chiral basis gamma_mu gamma_nu = diag(P_mu P_nu^dag, P_mu^dag P_nu),
// so C, A = (4 + m0) - C and A^{-1} split into two Hermitian 6x6 blocks per site.
//
// All of it is set-up work done once per gauge field, in FP64: kernel 1 forms the
// six F_mu,nu per site, kernel 2 assembles each 6x6 block, packs it (6 real
// diagonal + 15 complex lower entries) and inverts it by Gauss-Jordan elimination
// with partial pivoting, flagging a pivot below 1e-14 times the block's largest
// entry. The time boundary factor folded into the packed U_0 cancels in every
// plaquette (each temporal link there appears once plainly and once daggered).
#include "kernels.h"

namespace lqcd {

struct M3 {
  double2 e[9];
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // a * conj(b)
  return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// A * B, A * B^dag, A^dag * B
__device__ M3 mm(const M3& a, const M3& b) {
  M3 c;
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) {
      double2 s = make_double2(0, 0);
      for (int j = 0; j < 3; ++j) {
        double2 t = cmul(a.e[3 * i + j], b.e[3 * j + k]);
        s.x += t.x; s.y += t.y;
      }
      c.e[3 * i + k] = s;
    }
  return c;
}
__device__ M3 mmd(const M3& a, const M3& b) {
  M3 c;
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) {
      double2 s = make_double2(0, 0);
      for (int j = 0; j < 3; ++j) {
        double2 t = cmulc(a.e[3 * i + j], b.e[3 * k + j]);
        s.x += t.x; s.y += t.y;
      }
      c.e[3 * i + k] = s;
    }
  return c;
}
__device__ M3 mdm(const M3& a, const M3& b) {
  M3 c;
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) {
      double2 s = make_double2(0, 0);
      for (int j = 0; j < 3; ++j) {
        double2 t = cmulc(b.e[3 * j + k], a.e[3 * j + i]);  // conj(a_ji) b_jk
        s.x += t.x; s.y += t.y;
      }
      c.e[3 * i + k] = s;
    }
  return c;
}

struct Site4 {
  int v[4];
};

__device__ __forceinline__ int eo_index(const Geom& g, const Site4& s) {
  const int lex = ((s.v[0] * g.Z + s.v[1]) * g.Y + s.v[2]) * g.X + s.v[3];
  const int p = (s.v[0] + s.v[1] + s.v[2] + s.v[3]) & 1;
  return p * g.Vh + (lex >> 1);
}

__device__ __forceinline__ Site4 shifted(const Geom& g, Site4 s, int mu, int d) {
  const int ext[4] = {g.T, g.Z, g.Y, g.X};
  s.v[mu] = (s.v[mu] + d + ext[mu]) % ext[mu];
  return s;
}

__device__ M3 load_link(const Geom& g, const double2* links, int mu, const Site4& s) {
  M3 m;
  const int i = eo_index(g, s);
  for (int e = 0; e < 9; ++e) m.e[e] = links[(int64_t)(mu * 9 + e) * g.V + i];
  return m;
}

__constant__ int kPlaneMu[6] = {0, 0, 0, 1, 1, 2};
__constant__ int kPlaneNu[6] = {1, 2, 3, 2, 3, 3};

// F_mu,nu(x) = Q_mu,nu(x) - Q_mu,nu(x)^dag, one thread per (site, plane).
__global__ void clover_leaf_kernel(Geom g, const double2* __restrict__ links, double2* __restrict__ F) {
  const int64_t total = (int64_t)6 * g.V;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q % g.V);
    const int pl = (int)(q / g.V);
    const int mu = kPlaneMu[pl], nu = kPlaneNu[pl];
    const int p = i >= g.Vh ? 1 : 0;
    const Coord c = site_coords(g, p, i - p * g.Vh);
    Site4 x;
    x.v[0] = c.t; x.v[1] = c.z; x.v[2] = c.y; x.v[3] = c.x;
    const Site4 xpm = shifted(g, x, mu, 1), xpn = shifted(g, x, nu, 1);
    const Site4 xmm = shifted(g, x, mu, -1), xmn = shifted(g, x, nu, -1);
    const Site4 xmm_pn = shifted(g, xmm, nu, 1), xmm_mn = shifted(g, xmm, nu, -1);
    const Site4 xmn_pm = shifted(g, xmn, mu, 1);
    // leaf 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
    M3 q1 = mmd(mmd(mm(load_link(g, links, mu, x), load_link(g, links, nu, xpm)),
                    load_link(g, links, mu, xpn)),
                load_link(g, links, nu, x));
    // leaf 2: U_nu(x) U_mu(x-mu+nu)^dag U_nu(x-mu)^dag U_mu(x-mu)
    M3 q2 = mm(mmd(mmd(load_link(g, links, nu, x), load_link(g, links, mu, xmm_pn)),
                   load_link(g, links, nu, xmm)),
               load_link(g, links, mu, xmm));
    // leaf 3: U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
    // written as a^dag b with a = U_nu(x-mu-nu) U_mu(x-mu), b = U_mu(x-mu-nu) U_nu(x-nu)
    M3 q3 = mdm(mm(load_link(g, links, nu, xmm_mn), load_link(g, links, mu, xmm)),
                mm(load_link(g, links, mu, xmm_mn), load_link(g, links, nu, xmn)));
    // leaf 4: U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^dag
    M3 q4 = mmd(mm(mdm(load_link(g, links, nu, xmn), load_link(g, links, mu, xmn)),
                   load_link(g, links, nu, xmn_pm)),
                load_link(g, links, mu, x));
    for (int e = 0; e < 9; ++e) {
      const int r = e / 3, cc = e % 3;
      double2 s = make_double2(q1.e[e].x + q2.e[e].x + q3.e[e].x + q4.e[e].x,
                               q1.e[e].y + q2.e[e].y + q3.e[e].y + q4.e[e].y);
      const int et = 3 * cc + r;
      double2 st = make_double2(q1.e[et].x + q2.e[et].x + q3.e[et].x + q4.e[et].x,
                                q1.e[et].y + q2.e[et].y + q3.e[et].y + q4.e[et].y);
      // F = Q - Q^dag: F_rc = Q_rc - conj(Q_cr)
      F[((int64_t)pl * 9 + e) * g.V + i] = make_double2(s.x - st.x, s.y + st.y);
    }
  }
}

// 2x2 spin matrices P_mu (chiral basis gamma_mu = [[0, P_mu], [P_mu^dag, 0]]).
__device__ void spin_P(int mu, double2 P[4]) {
  for (int k = 0; k < 4; ++k) P[k] = make_double2(0, 0);
  if (mu == 0) { P[0] = make_double2(1, 0); P[3] = make_double2(1, 0); }
  if (mu == 1) { P[0] = make_double2(0, 1); P[3] = make_double2(0, -1); }
  if (mu == 2) { P[1] = make_double2(1, 0); P[2] = make_double2(-1, 0); }
  if (mu == 3) { P[1] = make_double2(0, 1); P[2] = make_double2(0, 1); }
}

// Packed-block helpers: 36 reals per chiral half = diag[6], then L(l,j) l>j (re, im).
__device__ __forceinline__ int lower_idx(int l, int j) { return 6 + 2 * (l * (l - 1) / 2 + j); }

// One thread per (site, chiral half h): assemble, pack, invert, pack.
__global__ void clover_block_kernel(Geom g, double m0, double c_sw, const double2* __restrict__ F,
                                    double* __restrict__ blk, double* __restrict__ inv, int* err) {
  const int64_t total = (int64_t)2 * g.V;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q % g.V);
    const int h = (int)(q / g.V);
    double2 M[36];
    for (int k = 0; k < 36; ++k) M[k] = make_double2(0, 0);
    for (int d = 0; d < 6; ++d) M[7 * d].x = 4.0 + m0;
    const double coef = -c_sw / 16.0;  // A = (4 + m0) - (c_sw/16) sum gamma gamma (x) F
    for (int pl = 0; pl < 6; ++pl) {
      const int mu = kPlaneMu[pl], nu = kPlaneNu[pl];
      double2 Pm[4], Pn[4], S[4];
      spin_P(mu, Pm);
      spin_P(nu, Pn);
      // h = 0: S = P_mu P_nu^dag ; h = 1: S = P_mu^dag P_nu
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          double2 s = make_double2(0, 0);
          for (int c = 0; c < 2; ++c) {
            double2 t = (h == 0) ? cmulc(Pm[2 * a + c], Pn[2 * b + c])        // Pm_ac conj(Pn_bc)
                                 : cmulc(Pn[2 * c + b], Pm[2 * c + a]);       // conj(Pm_ca) Pn_cb
            s.x += t.x; s.y += t.y;
          }
          S[2 * a + b] = s;
        }
      double2 f[9];
      for (int e = 0; e < 9; ++e) f[e] = F[((int64_t)pl * 9 + e) * g.V + i];
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
          for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
              double2 t = cmul(S[2 * a + b], f[3 * r + c]);
              M[(3 * a + r) * 6 + 3 * b + c].x += coef * t.x;
              M[(3 * a + r) * 6 + 3 * b + c].y += coef * t.y;
            }
    }
    // pack A
    double* out = blk;  // SoA of double2 chunks: chunk k of site i at (k * V + i) * 2
    double packed[36];
    double amax = 0.0;
    for (int l = 0; l < 6; ++l) {
      packed[l] = M[7 * l].x;
      for (int j = 0; j < l; ++j) {
        packed[lower_idx(l, j)] = M[6 * l + j].x;
        packed[lower_idx(l, j) + 1] = M[6 * l + j].y;
      }
    }
    for (int k = 0; k < 36; ++k) amax = fmax(amax, fabs(M[k].x) + fabs(M[k].y));
    for (int k = 0; k < 18; ++k) {
      const int64_t idx = ((int64_t)(18 * h + k) * g.V + i) * 2;
      out[idx] = packed[2 * k];
      out[idx + 1] = packed[2 * k + 1];
    }
    // Gauss-Jordan with partial pivoting on [M | I]
    double2 R[36];
    for (int k = 0; k < 36; ++k) R[k] = make_double2(k % 7 == 0 ? 1.0 : 0.0, 0.0);
    bool singular = false;
    for (int col = 0; col < 6; ++col) {
      int piv = col;
      double best = hypot(M[6 * col + col].x, M[6 * col + col].y);
      for (int r = col + 1; r < 6; ++r) {
        const double v = hypot(M[6 * r + col].x, M[6 * r + col].y);
        if (v > best) { best = v; piv = r; }
      }
      if (!(best > 1e-14 * amax)) { singular = true; break; }
      if (piv != col)
        for (int k = 0; k < 6; ++k) {
          double2 t = M[6 * col + k]; M[6 * col + k] = M[6 * piv + k]; M[6 * piv + k] = t;
          t = R[6 * col + k]; R[6 * col + k] = R[6 * piv + k]; R[6 * piv + k] = t;
        }
      const double2 d = M[6 * col + col];
      const double den = d.x * d.x + d.y * d.y;
      const double2 dinv = make_double2(d.x / den, -d.y / den);
      for (int k = 0; k < 6; ++k) {
        M[6 * col + k] = cmul(M[6 * col + k], dinv);
        R[6 * col + k] = cmul(R[6 * col + k], dinv);
      }
      for (int r = 0; r < 6; ++r) {
        if (r == col) continue;
        const double2 fct = M[6 * r + col];
        if (fct.x == 0.0 && fct.y == 0.0) continue;
        for (int k = 0; k < 6; ++k) {
          double2 t = cmul(fct, M[6 * col + k]);
          M[6 * r + k].x -= t.x; M[6 * r + k].y -= t.y;
          t = cmul(fct, R[6 * col + k]);
          R[6 * r + k].x -= t.x; R[6 * r + k].y -= t.y;
        }
      }
    }
    if (singular) {
      atomicOr(err, DEV_ERR_SINGULAR);
      for (int k = 0; k < 36; ++k) R[k] = make_double2(0, 0);
    }
    // pack the Hermitian part of the inverse
    for (int l = 0; l < 6; ++l) {
      packed[l] = R[7 * l].x;
      for (int j = 0; j < l; ++j) {
        packed[lower_idx(l, j)] = 0.5 * (R[6 * l + j].x + R[6 * j + l].x);
        packed[lower_idx(l, j) + 1] = 0.5 * (R[6 * l + j].y - R[6 * j + l].y);
      }
    }
    for (int k = 0; k < 18; ++k) {
      const int64_t idx = ((int64_t)(18 * h + k) * g.V + i) * 2;
      inv[idx] = packed[2 * k];
      inv[idx + 1] = packed[2 * k + 1];
    }
  }
}

// FP64 SoA double2 chunks [36][V] -> FP32 SoA float4 chunks [18][V].
__global__ void blocks_to_f32_kernel(Geom g, const double* __restrict__ b64, float* __restrict__ b32) {
  const int64_t total = (int64_t)18 * g.V;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q % g.V);
    const int k = (int)(q / g.V);
    const double2 a = reinterpret_cast<const double2*>(b64)[(int64_t)(2 * k) * g.V + i];
    const double2 b = reinterpret_cast<const double2*>(b64)[(int64_t)(2 * k + 1) * g.V + i];
    reinterpret_cast<float4*>(b32)[(int64_t)k * g.V + i] =
        make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
  }
}

static int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  const int64_t cap = 65535LL * 8;
  return (int)(b > cap ? cap : (b < 1 ? 1 : b));
}

cudaError_t launch_clover_build(const Geom& g, const void* links64, double m0, double c_sw,
                                void* leaf_tmp, void* blk64, void* inv64, void* blk32, void* inv32,
                                int* err_flag, cudaStream_t stream) {
  const int threads = 128;
  clover_leaf_kernel<<<grid_for((int64_t)6 * g.V, threads), threads, 0, stream>>>(
      g, (const double2*)links64, (double2*)leaf_tmp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  clover_block_kernel<<<grid_for((int64_t)2 * g.V, threads), threads, 0, stream>>>(
      g, m0, c_sw, (const double2*)leaf_tmp, (double*)blk64, (double*)inv64, err_flag);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  blocks_to_f32_kernel<<<grid_for((int64_t)18 * g.V, 256), 256, 0, stream>>>(g, (const double*)blk64,
                                                                               (float*)blk32);
  blocks_to_f32_kernel<<<grid_for((int64_t)18 * g.V, 256), 256, 0, stream>>>(g, (const double*)inv64,
                                                                               (float*)inv32);
  return cudaGetLastError();
}

// Packed FP64 blocks -> canonical [V][12][12] complex128 (site order), zero off the chiral blocks.
__global__ void blocks_export_kernel(Geom g, const double* __restrict__ b64, double2* __restrict__ out) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < g.V;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int lex = (int)q;
    int r = lex;
    const int x = r % g.X; r /= g.X;
    const int y = r % g.Y; r /= g.Y;
    const int z = r % g.Z;
    const int t = r / g.Z;
    const int i = ((t + z + y + x) & 1) * g.Vh + (lex >> 1);
    double2* o = out + (int64_t)lex * 144;
    for (int k = 0; k < 144; ++k) o[k] = make_double2(0, 0);
    for (int h = 0; h < 2; ++h) {
      double m[36];
      for (int k = 0; k < 18; ++k) {
        const int64_t idx = ((int64_t)(18 * h + k) * g.V + i) * 2;
        m[2 * k] = b64[idx];
        m[2 * k + 1] = b64[idx + 1];
      }
      for (int l = 0; l < 6; ++l) {
        o[(6 * h + l) * 12 + 6 * h + l] = make_double2(m[l], 0.0);
        for (int j = 0; j < l; ++j) {
          const double re = m[lower_idx(l, j)], im = m[lower_idx(l, j) + 1];
          o[(6 * h + l) * 12 + 6 * h + j] = make_double2(re, im);
          o[(6 * h + j) * 12 + 6 * h + l] = make_double2(re, -im);
        }
      }
    }
  }
}

cudaError_t launch_blocks_export(const Geom& g, const void* blk64, void* out, cudaStream_t stream) {
  blocks_export_kernel<<<grid_for(g.V, 128), 128, 0, stream>>>(g, (const double*)blk64, (double2*)out);
  return cudaGetLastError();
}

}  // namespace lqcd
