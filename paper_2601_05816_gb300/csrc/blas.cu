// Multi-rhs vector kernels of the batched GMRES (Algorithm 2) on packed blocks.
//
// A packed block of n complex numbers holds nrhs right-hand sides interleaved
// with the rhs index innermost, so element e belongs to rhs e % nrhs. Every
// streaming kernel runs a thread count that is a multiple of nrhs and strides
// by a multiple of nrhs, so each thread owns one rhs and keeps per-rhs partial
// sums in registers: the lane separation of the paper's Layout-2 dot product
// (Sec. V-B, Fig. 7) is delayed to the very end, where a block reduction in
// FP64 and a fixed-order cross-block sum (reduce_partials) produce one value
// per (vector, rhs). The summation order depends only on the launch shape, so
// results are bitwise reproducible run to run.
#include "kernels.h"

namespace lqcd {

BlasPlan blas_plan(int64_t n, int nrhs, int num_sms) {
  BlasPlan p;
  p.nrhs = nrhs;
  p.num_sms = num_sms;
  p.threads = nrhs * (256 / nrhs);
  int64_t want = (n + p.threads - 1) / p.threads;
  int64_t cap = 2 * (int64_t)num_sms;
  p.blocks = (int)(want < cap ? (want < 1 ? 1 : want) : cap);
  // the warp-split Gram-Schmidt kernel: epl = 2 when two elements per lane are possible
  // (even nrhs <= 64; taken by BF16 storage, and by FP32 above nrhs = 32), else one
  // (nrhs <= 32)
  p.epl = (nrhs % 2 == 0 && nrhs <= 64) ? 2 : 1;
  p.split = (p.epl == 2 || nrhs <= 32) ? 1 : 0;
  if (p.split) {
    const int64_t rows_per_tile = (32 * 2 / nrhs) * 2;   // a lower bound over the kernel shapes
    const int64_t tiles = (n / nrhs + rows_per_tile - 1) / rows_per_tile;
    const int64_t scap = 4 * (int64_t)num_sms;
    p.blocks = (int)(tiles < scap ? (tiles < 1 ? 1 : tiles) : scap);
  }
  return p;
}

template <typename C> struct RealOf;
template <> struct RealOf<float2> { using T = float; };
template <> struct RealOf<double2> { using T = double; };

// Basis storage -> compute type, and back (BF16 storage computes in FP32; rounding to nearest even).
__device__ __forceinline__ float2 to_c(float2 v) { return v; }
__device__ __forceinline__ double2 to_c(double2 v) { return v; }
__device__ __forceinline__ float2 to_c(__nv_bfloat162 v) { return __bfloat1622float2(v); }
// Read-only load of a basis element. A BF16 pair is read as one 32-bit word and
// widened with shifts (a BF16 value is the upper half of the FP32 bit pattern).
template <typename C>
__device__ __forceinline__ C ld_basis(const C* p) { return __ldg(p); }
__device__ __forceinline__ float2 ld_basis(const __nv_bfloat162* p) {
  const unsigned u = __ldg(reinterpret_cast<const unsigned*>(p));
  return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}
__device__ __forceinline__ void store_as(float2* p, float2 v) { *p = v; }
__device__ __forceinline__ void store_as(double2* p, double2 v) { *p = v; }
__device__ __forceinline__ void store_as(__nv_bfloat162* p, float2 v) { *p = __float22bfloat162_rn(v); }

// Block reduction of per-thread values (one per slot) into partials[blockIdx][slot][rhs].
template <int NS>
__device__ __forceinline__ void block_reduce_slots(const double (&vr)[NS], const double (&vi)[NS],
                                                   int nslots, int nrhs, double2* partials) {
  __shared__ double2 red[256];
  const int tid = threadIdx.x;
  const int per = blockDim.x / nrhs;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    if (s >= nslots) break;
    red[tid] = make_double2(vr[s], vi[s]);
    __syncthreads();
    if (tid < nrhs) {
      double2 acc = make_double2(0.0, 0.0);
      for (int q = 0; q < per; ++q) {
        const double2 v = red[tid + q * nrhs];
        acc.x += v.x;
        acc.y += v.y;
      }
      partials[((int64_t)blockIdx.x * nslots + s) * nrhs + tid] = acc;
    }
    __syncthreads();
  }
}

// Fixed-order sum of partials[blk][q] over blk for q < nq; one warp per q.
__global__ void reduce_partials_kernel(int nblk, int nq, const double2* __restrict__ partials,
                                       double2* __restrict__ out, const int* skip) {
  if (skip != nullptr && *skip != 0) return;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nq) return;
  double sx = 0.0, sy = 0.0;
  for (int b = lane; b < nblk; b += 32) {
    const double2 v = partials[(int64_t)b * nq + warp];
    sx += v.x;
    sy += v.y;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, off);
    sy += __shfl_xor_sync(0xffffffffu, sy, off);
  }
  if (lane == 0) out[warp] = make_double2(sx, sy);
}

static cudaError_t launch_reduce(int nblk, int nq, const void* partials, void* out, const int* skip,
                                 cudaStream_t stream) {
  const int threads = 256;
  const int blocks = (nq * 32 + threads - 1) / threads;
  reduce_partials_kernel<<<blocks, threads, 0, stream>>>(nblk, nq, (const double2*)partials,
                                                          (double2*)out, skip);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ Gram-Schmidt pass

template <typename C, int NVB, bool UPDATE, bool DOTS, bool NORM>
__global__ void __launch_bounds__(256)
gs_pass_kernel(int64_t n, int nrhs, int nvec, const C* __restrict__ basis, int64_t vstride,
               C* __restrict__ w, const double2* __restrict__ coef, const double* __restrict__ oscale,
               double2* __restrict__ partials, const int* skip) {
  using Real = typename RealOf<C>::T;
  if (skip != nullptr && *skip != 0) return;
  const int tid = threadIdx.x;
  const int r = tid % nrhs;
  Real cr[NVB], ci[NVB], ar[NVB], ai[NVB];
#pragma unroll
  for (int i = 0; i < NVB; ++i) {
    ar[i] = 0; ai[i] = 0; cr[i] = 0; ci[i] = 0;
    if (UPDATE && i < nvec) {
      const double2 c = coef[(int64_t)i * nrhs + r];
      cr[i] = (Real)c.x;
      ci[i] = (Real)c.y;
    }
  }
  Real nn = 0;
  const Real o_scale = (UPDATE && oscale != nullptr) ? (Real)oscale[r] : (Real)1;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + tid; e < n; e += stride) {
    C wv = w[e];
    if (UPDATE) {
      C v[NVB];
#pragma unroll
      for (int i = 0; i < NVB; ++i)
        if (i < nvec) v[i] = __ldg(basis + i * vstride + e);
#pragma unroll
      for (int i = 0; i < NVB; ++i) {
        if (i < nvec) {
          wv.x -= cr[i] * v[i].x - ci[i] * v[i].y;
          wv.y -= cr[i] * v[i].y + ci[i] * v[i].x;
        }
      }
      w[e] = C{wv.x * o_scale, wv.y * o_scale};
      if (DOTS) {
#pragma unroll
        for (int i = 0; i < NVB; ++i) {
          if (i < nvec) {
            ar[i] += v[i].x * wv.x + v[i].y * wv.y;
            ai[i] += v[i].x * wv.y - v[i].y * wv.x;
          }
        }
      }
    } else if (DOTS) {
#pragma unroll
      for (int i = 0; i < NVB; ++i) {
        if (i < nvec) {
          const C v = __ldg(basis + i * vstride + e);
          ar[i] += v.x * wv.x + v.y * wv.y;
          ai[i] += v.x * wv.y - v.y * wv.x;
        }
      }
    }
    if (NORM) nn += wv.x * wv.x + wv.y * wv.y;
  }
  double vr[NVB + 1], vi[NVB + 1];
#pragma unroll
  for (int i = 0; i < NVB + 1; ++i) { vr[i] = 0.0; vi[i] = 0.0; }
#pragma unroll
  for (int i = 0; i < NVB; ++i)
    if (i < nvec) { vr[i] = DOTS ? (double)ar[i] : 0.0; vi[i] = DOTS ? (double)ai[i] : 0.0; }
  // norm goes to slot nvec
#pragma unroll
  for (int i = 0; i < NVB + 1; ++i)
    if (i == nvec) { vr[i] = NORM ? (double)nn : 0.0; vi[i] = 0.0; }
  block_reduce_slots<NVB + 1>(vr, vi, nvec + 1, nrhs, partials);
}

// Warp-split Gram-Schmidt pass. The block vector is viewed as rows of nrhs
// elements (the packed layout puts the rhs innermost); each lane owns EPL
// consecutive elements of a row (EPL = 2: one 16-byte FP32 or 8-byte BF16 load
// per vector, so every warp load moves 256 B of FP32 / 128-256 B of BF16) and so
// a fixed set of EPL rhs; a warp covers H = 32 * EPL / nrhs rows at once. All
// eight warps of a CTA walk the same element tiles of 32 * U "slots" (each slot
// EPL elements), and warp k owns the basis vectors i = k, k + 8, ...: its loads
// of those vectors stay in registers, and the loads of the next tile are issued
// before the current one is processed (register double buffering). For an update
// each warp puts its partial sum_i c_i v_i in shared memory and the first 32 * U
// threads ("slot threads", one per slot) form w - sum in one fixed summation
// order and store it; the updated tile goes through shared memory to every warp
// for the dot products. Registers stay low (several CTAs per SM).
// One lane's EPL basis elements as loaded (storage format): the prefetched tile is
// held in this form, so a BF16 tile in flight costs half the registers of FP32.
template <typename B, int EPL> struct RawT;
template <> struct RawT<float2, 1> { using T = float2; };
template <> struct RawT<float2, 2> { using T = float4; };
template <> struct RawT<double2, 1> { using T = double2; };
template <> struct RawT<__nv_bfloat162, 1> { using T = unsigned; };
template <> struct RawT<__nv_bfloat162, 2> { using T = uint2; };

__device__ __forceinline__ void ld_raw(const float2* p, float2& o) { o = __ldg(p); }
__device__ __forceinline__ void ld_raw(const float2* p, float4& o) { o = __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void ld_raw(const double2* p, double2& o) { o = __ldg(p); }
__device__ __forceinline__ void ld_raw(const __nv_bfloat162* p, unsigned& o) {
  o = __ldg(reinterpret_cast<const unsigned*>(p));
}
__device__ __forceinline__ void ld_raw(const __nv_bfloat162* p, uint2& o) {
  o = __ldg(reinterpret_cast<const uint2*>(p));
}
// BF16 -> FP32 is exact: the BF16 bits are the upper half of the FP32 pattern
__device__ __forceinline__ float2 bf2_to_f2(unsigned u) {
  return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}
__device__ __forceinline__ void unpack_raw(const float2& r, float2 (&o)[1]) { o[0] = r; }
__device__ __forceinline__ void unpack_raw(const float4& r, float2 (&o)[2]) {
  o[0] = make_float2(r.x, r.y);
  o[1] = make_float2(r.z, r.w);
}
__device__ __forceinline__ void unpack_raw(const double2& r, double2 (&o)[1]) { o[0] = r; }
__device__ __forceinline__ void unpack_raw(const unsigned& r, float2 (&o)[1]) { o[0] = bf2_to_f2(r); }
__device__ __forceinline__ void unpack_raw(const uint2& r, float2 (&o)[2]) {
  o[0] = bf2_to_f2(r.x);
  o[1] = bf2_to_f2(r.y);
}

// plain (coherent) loads of w, which the same kernel may have written in an earlier pass
template <int EPL>
__device__ __forceinline__ void ld_w(const float2* p, float2 (&o)[EPL]) {
  if constexpr (EPL == 2) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = make_float2(v.x, v.y);
    o[1] = make_float2(v.z, v.w);
  } else {
    o[0] = *p;
  }
}
template <int EPL>
__device__ __forceinline__ void ld_w(const double2* p, double2 (&o)[EPL]) {
#pragma unroll
  for (int q = 0; q < EPL; ++q) o[q] = p[q];
}
template <int EPL>
__device__ __forceinline__ void st_w(float2* p, const float2 (&v)[EPL]) {
  if constexpr (EPL == 2) *reinterpret_cast<float4*>(p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
  else *p = v[0];
}
template <int EPL>
__device__ __forceinline__ void st_w(double2* p, const double2 (&v)[EPL]) {
#pragma unroll
  for (int q = 0; q < EPL; ++q) p[q] = v[q];
}
template <int EPL>
__device__ __forceinline__ void st_w(__nv_bfloat162* p, const float2 (&v)[EPL]) {
  if constexpr (EPL == 2) {
    const __nv_bfloat162 a = __float22bfloat162_rn(v[0]), b = __float22bfloat162_rn(v[1]);
    uint2 u;
    memcpy(&u.x, &a, 4);
    memcpy(&u.y, &b, 4);
    *reinterpret_cast<uint2*>(p) = u;
  } else {
    *p = __float22bfloat162_rn(v[0]);
  }
}

template <typename C, typename B, int NVW, int U, int EPL, bool UPDATE, bool DOTS, bool NORM>
__global__ void __launch_bounds__(256)
gs_split_kernel(int64_t n, int nrhs, int nvec, const B* __restrict__ basis, int64_t vstride,
                C* __restrict__ w, const double2* __restrict__ coef, const double* __restrict__ oscale,
                B* __restrict__ wout, double2* __restrict__ partials, const int* skip) {
  using Real = typename RealOf<C>::T;
  static_assert(32 * U <= 256, "one slot thread per tile slot");
  if (skip != nullptr && *skip != 0) return;
  __shared__ C part[8][32 * U * EPL];
  __shared__ C wsm[2][32 * U * EPL];
  __shared__ double2 red[8][EPL][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lanes_per_row = nrhs / EPL;
  const int H = 32 / lanes_per_row;
  const int r = (lane % lanes_per_row) * EPL;      // first rhs of this lane
  const int hrow = lane / lanes_per_row;
  const bool lane_on = hrow < H;
  const int64_t Q = n / nrhs;
  const int64_t tile_rows = (int64_t)H * U;
  // slot thread: slot s = threadIdx.x = u * 32 + l, row offset l / lanes_per_row + H u
  const int slot = threadIdx.x;
  const bool is_slot = slot < 32 * U;
  const int s_l = slot & 31, s_u = slot >> 5;
  const bool s_on = is_slot && (s_l / lanes_per_row) < H;
  const int s_r = (s_l % lanes_per_row) * EPL;
  // optional per-rhs factor applied to the updated w before it is stored
  Real s_scale[EPL];
#pragma unroll
  for (int q = 0; q < EPL; ++q)
    s_scale[q] = (UPDATE && oscale != nullptr && s_on) ? (Real)oscale[s_r + q] : (Real)1;
  Real cr[NVW][EPL], ci[NVW][EPL], ar[NVW][EPL], ai[NVW][EPL];
#pragma unroll
  for (int k = 0; k < NVW; ++k)
#pragma unroll
    for (int q = 0; q < EPL; ++q) {
      cr[k][q] = 0; ci[k][q] = 0; ar[k][q] = 0; ai[k][q] = 0;
      const int i = warp + 8 * k;
      if (UPDATE && lane_on && i < nvec) {
        const double2 c = coef[(int64_t)i * nrhs + r + q];
        cr[k][q] = (Real)c.x;
        ci[k][q] = (Real)c.y;
      }
    }
  Real nn[EPL];
#pragma unroll
  for (int q = 0; q < EPL; ++q) nn[q] = 0;
  using R = typename RawT<B, EPL>::T;
  C v[NVW][U][EPL];
  R vn[NVW][U];
  C w_old[EPL], wn[EPL];
  auto load_tile = [&](int64_t t, R (&vv)[NVW][U], C (&ww)[EPL]) {
    const int64_t row0 = t * tile_rows;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t row = row0 + hrow + (int64_t)H * u;
      const bool ok = lane_on && row < Q;
      const int64_t e = row * nrhs + r;
#pragma unroll
      for (int k = 0; k < NVW; ++k) {
        const int i = warp + 8 * k;
        if (i < nvec && ok) ld_raw(basis + i * vstride + e, vv[k][u]);
        else vv[k][u] = R{};
      }
    }
    const int64_t s_row = row0 + s_l / lanes_per_row + (int64_t)H * s_u;
    if (s_on && s_row < Q) {
      ld_w<EPL>(w + s_row * nrhs + s_r, ww);
    } else {
#pragma unroll
      for (int q = 0; q < EPL; ++q) ww[q] = C{0, 0};
    }
  };
  int parity = 0;
  int64_t t = blockIdx.x;
  if (t * tile_rows < Q) load_tile(t, vn, wn);
  for (; t * tile_rows < Q; t += gridDim.x, parity ^= 1) {
#pragma unroll
    for (int k = 0; k < NVW; ++k)
#pragma unroll
      for (int u = 0; u < U; ++u) unpack_raw(vn[k][u], v[k][u]);
#pragma unroll
    for (int q = 0; q < EPL; ++q) w_old[q] = wn[q];
    if ((t + gridDim.x) * tile_rows < Q) load_tile(t + gridDim.x, vn, wn);
    const int64_t row0 = t * tile_rows;
    const int64_t s_row = row0 + s_l / lanes_per_row + (int64_t)H * s_u;
    const bool s_ok = s_on && s_row < Q;
    const int64_t s_e = s_row * nrhs + s_r;
    if (UPDATE) {
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int q = 0; q < EPL; ++q) {
          Real pr = 0, pi = 0;
#pragma unroll
          for (int k = 0; k < NVW; ++k) {
            pr += cr[k][q] * v[k][u][q].x - ci[k][q] * v[k][u][q].y;
            pi += cr[k][q] * v[k][u][q].y + ci[k][q] * v[k][u][q].x;
          }
          part[warp][(u * 32 + lane) * EPL + q] = C{pr, pi};
        }
      __syncthreads();
      if (is_slot) {
        C w_new[EPL], ws[EPL];
#pragma unroll
        for (int q = 0; q < EPL; ++q) {
          Real sr = 0, si = 0;
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            const C pq = part[p][slot * EPL + q];
            sr += pq.x;
            si += pq.y;
          }
          w_new[q] = C{w_old[q].x - sr, w_old[q].y - si};
          ws[q] = C{w_new[q].x * s_scale[q], w_new[q].y * s_scale[q]};
          wsm[parity][slot * EPL + q] = w_new[q];
          if (NORM) nn[q] += w_new[q].x * w_new[q].x + w_new[q].y * w_new[q].y;
        }
        if (s_ok) {
          if (wout != nullptr) st_w<EPL>(wout + s_e, ws);  // the normalised vector goes to the basis
          else st_w<EPL>(w + s_e, ws);
        }
      }
    } else if (is_slot) {
#pragma unroll
      for (int q = 0; q < EPL; ++q) {
        wsm[parity][slot * EPL + q] = w_old[q];
        if (NORM) nn[q] += w_old[q].x * w_old[q].x + w_old[q].y * w_old[q].y;
      }
    }
    __syncthreads();
    if (DOTS) {
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int q = 0; q < EPL; ++q) {
          const C wv = wsm[parity][(u * 32 + lane) * EPL + q];
#pragma unroll
          for (int k = 0; k < NVW; ++k) {
            ar[k][q] += v[k][u][q].x * wv.x + v[k][u][q].y * wv.y;
            ai[k][q] += v[k][u][q].x * wv.y - v[k][u][q].y * wv.x;
          }
        }
    }
  }
  // per-(vector, rhs) sums over the lanes of a warp that share the rhs: rhs R sits in
  // element q = R % EPL of the lanes (R / EPL) + h * lanes_per_row, h < H
  const int nslots = nvec + 1;
#pragma unroll
  for (int k = 0; k < NVW; ++k) {
#pragma unroll
    for (int q = 0; q < EPL; ++q)
      red[warp][q][lane] = make_double2(DOTS ? (double)ar[k][q] : 0.0, DOTS ? (double)ai[k][q] : 0.0);
    __syncwarp();
    const int i = warp + 8 * k;
    // nrhs can exceed 32 with EPL = 2: a lane then writes rhs lane and lane + 32
    for (int R = lane; R < nrhs && i < nvec; R += 32) {
      const int q = R % EPL, l0 = R / EPL;
      double2 acc = make_double2(0.0, 0.0);
      for (int h = 0; h < H; ++h) {
        acc.x += red[warp][q][l0 + h * lanes_per_row].x;
        acc.y += red[warp][q][l0 + h * lanes_per_row].y;
      }
      partials[((int64_t)blockIdx.x * nslots + i) * nrhs + R] = acc;
    }
    __syncwarp();
  }
  // the norm is held by the slot threads (warps 0 .. U-1)
  __syncthreads();
#pragma unroll
  for (int q = 0; q < EPL; ++q) red[warp][q][lane] = make_double2(NORM && is_slot ? (double)nn[q] : 0.0, 0.0);
  __syncthreads();
  if (threadIdx.x < nrhs) {
    const int q = threadIdx.x % EPL, l0 = threadIdx.x / EPL;
    double acc = 0.0;
    for (int u = 0; u < U; ++u)
      for (int h = 0; h < H; ++h) acc += red[u][q][l0 + h * lanes_per_row].x;
    partials[((int64_t)blockIdx.x * nslots + nvec) * nrhs + threadIdx.x] = make_double2(acc, 0.0);
  }
}

template <typename C, typename B, int NVW, int U, int EPL>
static void gs_split_dispatch(int blocks, int64_t n, int nrhs, int nvec, const void* basis, int64_t vstride,
                              void* w, const void* coef, const double* oscale, void* wout, bool update, bool dots,
                              bool norm, void* partials, const int* skip, cudaStream_t stream) {
  const B* b = (const B*)basis;
  C* wp = (C*)w;
  B* wo = (B*)wout;
  const double2* cf = (const double2*)coef;
  double2* pa = (double2*)partials;
#define GSS_LAUNCH(UP, D, N)                                                                             \
  gs_split_kernel<C, B, NVW, U, EPL, UP, D, N><<<blocks, 256, 0, stream>>>(n, nrhs, nvec, b, vstride, wp, cf, \
                                                                      oscale, wo, pa, skip)
  if (update) {
    if (dots) { if (norm) GSS_LAUNCH(true, true, true); else GSS_LAUNCH(true, true, false); }
    else { if (norm) GSS_LAUNCH(true, false, true); else GSS_LAUNCH(true, false, false); }
  } else {
    if (dots) { if (norm) GSS_LAUNCH(false, true, true); else GSS_LAUNCH(false, true, false); }
    else GSS_LAUNCH(false, false, true);
  }
#undef GSS_LAUNCH
}

template <typename C, int NVB>
static void gs_dispatch(const BlasPlan& p, int64_t n, int nvec, const void* basis, int64_t vstride,
                        void* w, const void* coef, const double* oscale, bool update, bool dots, bool norm,
                        void* partials, const int* skip, cudaStream_t stream) {
  const C* b = (const C*)basis;
  C* wp = (C*)w;
  const double2* cf = (const double2*)coef;
  double2* pa = (double2*)partials;
#define GS_LAUNCH(U, D, N) \
  gs_pass_kernel<C, NVB, U, D, N><<<p.blocks, p.threads, 0, stream>>>(n, p.nrhs, nvec, b, vstride, wp, cf, oscale, pa, skip)
  if (update) {
    if (dots) { if (norm) GS_LAUNCH(true, true, true); else GS_LAUNCH(true, true, false); }
    else { if (norm) GS_LAUNCH(true, false, true); else GS_LAUNCH(true, false, false); }
  } else {
    if (dots) { if (norm) GS_LAUNCH(false, true, true); else GS_LAUNCH(false, true, false); }
    else GS_LAUNCH(false, false, true);
  }
#undef GS_LAUNCH
}

cudaError_t launch_gs_pass(bool f64, const BlasPlan& plan, int64_t n, int nvec, const void* basis,
                           int64_t vstride, void* w, const void* coef, bool update, bool dots,
                           bool norm, void* partials, void* out, const int* skip,
                           cudaStream_t stream, const double* oscale, bool basis_bf16, void* wout) {
  if (nvec < 1 || nvec > 64) return cudaErrorInvalidValue;
  if (basis_bf16 && (f64 || !plan.split)) return cudaErrorInvalidValue;
  if (!f64) {
    int used = 0;
    const cudaError_t e =
        basis_bf16 ? launch_gs_stream_bf16(plan, n, nvec, basis, vstride, w, coef, update, dots, norm, partials,
                                           skip, stream, oscale, wout, &used)
                   : launch_gs_stream_f32(plan, n, nvec, basis, vstride, w, coef, update, dots, norm, partials,
                                          skip, stream, oscale, wout, &used);
    if (e == cudaSuccess) {
      if (!dots && !norm) return cudaSuccess;
      return launch_reduce(used, (nvec + 1) * plan.nrhs, partials, out, skip, stream);
    }
    if (e != cudaErrorNotSupported) return e;
  }
  // FP64 runs the split kernel with one element per lane, so only for nrhs <= 32
  if (plan.split && (!f64 || plan.nrhs <= 32)) {
  // Elements per lane: FP64 and FP32 take one (a 16- / 8-byte load per lane) up to
  // nrhs = 32, FP32 two above; BF16 takes two for even nrhs (8-byte loads). Tiles of
  // U slots keep about 2 KB of basis loads in flight per warp (U * NVW loads).
#define GSS_NVW(NW)                                                                                        \
  if (f64) gs_split_dispatch<double2, double2, NW, (NW >= 4 ? 1 : 4 / NW), 1>(plan.blocks, n, plan.nrhs, nvec, \
      basis, vstride, w, coef, oscale, wout, update, dots, norm, partials, skip, stream);                   \
  else if (basis_bf16 && plan.epl == 2) gs_split_dispatch<float2, __nv_bfloat162, NW, (NW >= 8 ? 1 : 8 / NW), 2>( \
      plan.blocks, n, plan.nrhs, nvec, basis, vstride, w, coef, oscale, wout, update, dots, norm, partials,    \
      skip, stream);                                                                                          \
  else if (basis_bf16) gs_split_dispatch<float2, __nv_bfloat162, NW, (NW >= 8 ? 1 : 8 / NW), 1>(plan.blocks,  \
      n, plan.nrhs, nvec, basis, vstride, w, coef, oscale, wout, update, dots, norm, partials, skip, stream);  \
  else if (plan.nrhs > 32) gs_split_dispatch<float2, float2, NW, (NW >= 4 ? 1 : 4 / NW), 2>(plan.blocks, n,  \
      plan.nrhs, nvec, basis, vstride, w, coef, oscale, wout, update, dots, norm, partials, skip, stream);   \
  else gs_split_dispatch<float2, float2, NW, (NW >= 8 ? 1 : 8 / NW), 1>(plan.blocks, n, plan.nrhs, nvec,     \
      basis, vstride, w, coef, oscale, wout, update, dots, norm, partials, skip, stream);
    if (nvec <= 8) { GSS_NVW(1) }
    else if (nvec <= 16) { GSS_NVW(2) }
    else if (nvec <= 32) { GSS_NVW(4) }
    else { GSS_NVW(8) }
#undef GSS_NVW
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (!dots && !norm) return cudaSuccess;
    return launch_reduce(plan.blocks, (nvec + 1) * plan.nrhs, partials, out, skip, stream);
  }
#define GS_NVB(NV)                                                                                \
  if (f64) gs_dispatch<double2, NV>(plan, n, nvec, basis, vstride, w, coef, oscale, update, dots, norm, \
                                    partials, skip, stream);                                            \
  else gs_dispatch<float2, NV>(plan, n, nvec, basis, vstride, w, coef, oscale, update, dots, norm,        \
                               partials, skip, stream);
  if (nvec <= 4) { GS_NVB(4) }
  else if (nvec <= 8) { GS_NVB(8) }
  else if (nvec <= 16) { GS_NVB(16) }
  else if (nvec <= 32) { GS_NVB(32) }
  else { GS_NVB(64) }
#undef GS_NVB
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (!dots && !norm) return cudaSuccess;
  return launch_reduce(plan.blocks, (nvec + 1) * plan.nrhs, partials, out, skip, stream);
}

// ------------------------------------------------------------------ small streaming kernels

template <typename T>
__global__ void __launch_bounds__(256)
sub_norm_kernel(int64_t n, int nrhs, const double2* __restrict__ b, const T* __restrict__ t,
                double2* __restrict__ r, double2* __restrict__ partials) {
  double nn = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    const double2 bv = b[e];
    const T tv = t[e];
    const double2 rv = make_double2(bv.x - (double)tv.x, bv.y - (double)tv.y);
    r[e] = rv;
    nn += rv.x * rv.x + rv.y * rv.y;
  }
  double vr[1] = {nn}, vi[1] = {0.0};
  block_reduce_slots<1>(vr, vi, 1, nrhs, partials);
}

cudaError_t launch_sub_norm(const BlasPlan& plan, int64_t n, const void* b, const void* t, void* r,
                            void* partials, void* out, cudaStream_t stream, bool t_f32) {
  if (t_f32)
    sub_norm_kernel<float2><<<plan.blocks, plan.threads, 0, stream>>>(
        n, plan.nrhs, (const double2*)b, (const float2*)t, (double2*)r, (double2*)partials);
  else
    sub_norm_kernel<double2><<<plan.blocks, plan.threads, 0, stream>>>(
        n, plan.nrhs, (const double2*)b, (const double2*)t, (double2*)r, (double2*)partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_reduce(plan.blocks, plan.nrhs, partials, out, nullptr, stream);
}

__global__ void __launch_bounds__(256)
diff_to_f32_kernel(int64_t n, const double2* __restrict__ a, const double2* __restrict__ b,
                   float2* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    const double2 av = a[e], bv = b[e];
    out[e] = make_float2((float)(av.x - bv.x), (float)(av.y - bv.y));
  }
}

cudaError_t launch_diff_to_f32(int64_t n, const void* a, const void* b, void* out, cudaStream_t stream) {
  const int threads = 256;
  int64_t blocks = (n + threads - 1) / threads;
  if (blocks > 65535 * 16) blocks = 65535 * 16;
  diff_to_f32_kernel<<<(int)blocks, threads, 0, stream>>>(n, (const double2*)a, (const double2*)b, (float2*)out);
  return cudaGetLastError();
}

template <typename C>
__global__ void __launch_bounds__(256)
norm2_kernel(int64_t n, int nrhs, const C* __restrict__ v, double2* __restrict__ partials) {
  double nn = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    const C x = v[e];
    nn += (double)x.x * x.x + (double)x.y * x.y;
  }
  double vr[1] = {nn}, vi[1] = {0.0};
  block_reduce_slots<1>(vr, vi, 1, nrhs, partials);
}

cudaError_t launch_norm2(bool f64, const BlasPlan& plan, int64_t n, const void* v, void* partials,
                         void* out, cudaStream_t stream) {
  if (f64)
    norm2_kernel<double2><<<plan.blocks, plan.threads, 0, stream>>>(n, plan.nrhs, (const double2*)v,
                                                                     (double2*)partials);
  else
    norm2_kernel<float2><<<plan.blocks, plan.threads, 0, stream>>>(n, plan.nrhs, (const float2*)v,
                                                                    (double2*)partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_reduce(plan.blocks, plan.nrhs, partials, out, nullptr, stream);
}

template <typename CD>
__global__ void scale_convert_kernel(int64_t n, int nrhs, const double2* __restrict__ src,
                                     const double* __restrict__ scale, CD* __restrict__ dst) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    const double s = scale[e % nrhs];
    const double2 v = src[e];
    CD o;
    o.x = v.x * s;
    o.y = v.y * s;
    dst[e] = o;
  }
}

static int stream_blocks(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  const int64_t cap = 152 * 16;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <>
__global__ void scale_convert_kernel<__nv_bfloat162>(int64_t n, int nrhs, const double2* __restrict__ src,
                                                     const double* __restrict__ scale,
                                                     __nv_bfloat162* __restrict__ dst) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    const double s = scale[e % nrhs];
    const double2 v = src[e];
    dst[e] = __float22bfloat162_rn(make_float2((float)(v.x * s), (float)(v.y * s)));
  }
}

cudaError_t launch_scale_convert(bool dst_f64, int64_t n, int nrhs, const void* src,
                                 const double* scale, void* dst, cudaStream_t stream, bool dst_bf16) {
  const int threads = 256;
  const int blocks = stream_blocks(n, threads);
  if (dst_bf16)
    scale_convert_kernel<__nv_bfloat162><<<blocks, threads, 0, stream>>>(n, nrhs, (const double2*)src, scale,
                                                                         (__nv_bfloat162*)dst);
  else if (dst_f64)
    scale_convert_kernel<double2><<<blocks, threads, 0, stream>>>(n, nrhs, (const double2*)src, scale,
                                                                  (double2*)dst);
  else
    scale_convert_kernel<float2><<<blocks, threads, 0, stream>>>(n, nrhs, (const double2*)src, scale,
                                                                 (float2*)dst);
  return cudaGetLastError();
}

template <typename C>
__global__ void scale_inplace_kernel(int64_t n, int nrhs, C* __restrict__ v,
                                     const double* __restrict__ scale, const int* skip) {
  if (skip != nullptr && *skip != 0) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    const double s = scale[e % nrhs];
    C x = v[e];
    x.x = x.x * s;
    x.y = x.y * s;
    v[e] = x;
  }
}

cudaError_t launch_scale_inplace(bool f64, int64_t n, int nrhs, void* v, const double* scale,
                                 const int* skip, cudaStream_t stream) {
  const int threads = 256;
  const int blocks = stream_blocks(n, threads);
  if (f64)
    scale_inplace_kernel<double2><<<blocks, threads, 0, stream>>>(n, nrhs, (double2*)v, scale, skip);
  else
    scale_inplace_kernel<float2><<<blocks, threads, 0, stream>>>(n, nrhs, (float2*)v, scale, skip);
  return cudaGetLastError();
}

// x += sum_i y[i][r] v_i with the sum formed in the basis precision (the
// correction of one restart cycle; its rounding is removed by the next FP64
// true residual) and added to x in FP64. A CTA owns tiles of EPT * blockDim.x
// consecutive elements and walks the vectors in the outer loop: per vector it reads
// one contiguous run of the tile (four vectors at a time: 4 EPT independent loads in flight per thread), with
// the partial sums of its EPT elements in registers. blockDim.x is a multiple of
// nrhs, so a thread's rhs (and its coefficients) are the same for all its elements.
template <typename C, typename B, int EPT>
__global__ void __launch_bounds__(256)
update_x_kernel(int64_t n, int nrhs, const B* __restrict__ basis, int64_t vstride,
                const double2* __restrict__ y, const int* __restrict__ kmax, double2* __restrict__ x) {
  using Real = typename RealOf<C>::T;
  extern __shared__ double2 ys[];
  const int k = *kmax;
  for (int q = threadIdx.x; q < k * nrhs; q += blockDim.x) ys[q] = y[q];
  __syncthreads();
  if (k == 0) return;
  const int r = threadIdx.x % nrhs;
  const int64_t tile = (int64_t)blockDim.x * EPT;
  for (int64_t base = (int64_t)blockIdx.x * tile; base < n; base += (int64_t)gridDim.x * tile) {
    Real sr[EPT], si[EPT];
#pragma unroll
    for (int u = 0; u < EPT; ++u) { sr[u] = 0; si[u] = 0; }
    // four vectors per step: their EPT loads each are independent, so 4 EPT are in flight
    int i = 0;
    for (; i + 4 <= k; i += 4) {
      C v[4][EPT];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const B* vi = basis + (i + q) * vstride + base + threadIdx.x;
#pragma unroll
        for (int u = 0; u < EPT; ++u)
          v[q][u] = base + threadIdx.x + (int64_t)u * blockDim.x < n ? C(ld_basis(vi + (int64_t)u * blockDim.x))
                                                                      : C{};
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double2 c = ys[(i + q) * nrhs + r];
        const Real crr = (Real)c.x, cii = (Real)c.y;
#pragma unroll
        for (int u = 0; u < EPT; ++u) {
          sr[u] += crr * v[q][u].x - cii * v[q][u].y;
          si[u] += crr * v[q][u].y + cii * v[q][u].x;
        }
      }
    }
    for (; i < k; ++i) {
      const double2 c = ys[i * nrhs + r];
      const Real crr = (Real)c.x, cii = (Real)c.y;
      const B* vi = basis + i * vstride + base + threadIdx.x;
#pragma unroll
      for (int u = 0; u < EPT; ++u) {
        if (base + threadIdx.x + (int64_t)u * blockDim.x < n) {
          const C v = C(ld_basis(vi + (int64_t)u * blockDim.x));
          sr[u] += crr * v.x - cii * v.y;
          si[u] += crr * v.y + cii * v.x;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int64_t e = base + threadIdx.x + (int64_t)u * blockDim.x;
      if (e < n) {
        double2 xv = x[e];
        xv.x += (double)sr[u];
        xv.y += (double)si[u];
        x[e] = xv;
      }
    }
  }
}

cudaError_t launch_update_x(bool basis_f64, int64_t n, int nrhs, int nvec_max, const void* basis,
                            int64_t vstride, const void* y, const int* kmax, void* x,
                            cudaStream_t stream, bool basis_bf16) {
  constexpr int EPT = 4;
  const int threads = nrhs * (256 / nrhs);
  int64_t tiles = (n + (int64_t)threads * EPT - 1) / ((int64_t)threads * EPT);
  const int blocks = (int)(tiles < 1 ? 1 : (tiles > 152 * 8 ? 152 * 8 : tiles));
  const size_t smem = sizeof(double2) * (size_t)nvec_max * nrhs;
  if (basis_bf16)
    update_x_kernel<float2, __nv_bfloat162, EPT><<<blocks, threads, smem, stream>>>(
        n, nrhs, (const __nv_bfloat162*)basis, vstride, (const double2*)y, kmax, (double2*)x);
  else if (basis_f64)
    update_x_kernel<double2, double2, EPT><<<blocks, threads, smem, stream>>>(
        n, nrhs, (const double2*)basis, vstride, (const double2*)y, kmax, (double2*)x);
  else
    update_x_kernel<float2, float2, EPT><<<blocks, threads, smem, stream>>>(
        n, nrhs, (const float2*)basis, vstride, (const double2*)y, kmax, (double2*)x);
  return cudaGetLastError();
}

template <typename CS, typename CD>
__global__ void convert_kernel(int64_t n, const CS* __restrict__ src, CD* __restrict__ dst) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    const CS v = src[e];
    CD o;
    o.x = v.x;
    o.y = v.y;
    dst[e] = o;
  }
}

cudaError_t launch_convert(bool to_f64, int64_t n, const void* src, void* dst, cudaStream_t stream) {
  const int threads = 256;
  const int blocks = stream_blocks(n, threads);
  if (to_f64)
    convert_kernel<float2, double2><<<blocks, threads, 0, stream>>>(n, (const float2*)src, (double2*)dst);
  else
    convert_kernel<double2, float2><<<blocks, threads, 0, stream>>>(n, (const double2*)src, (float2*)dst);
  return cudaGetLastError();
}

}  // namespace lqcd
