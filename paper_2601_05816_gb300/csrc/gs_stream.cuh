// Streaming Gram-Schmidt pass: warp-specialised, basis tiles staged in shared
// memory by bulk asynchronous copies (cp.async.bulk, completion on mbarriers).
//
// The pass is one pass of the orthogonalisation in Algorithm 2's Arnoldi step
// (Sec. III-A-2), done as classical Gram-Schmidt with re-orthogonalisation (CGS2,
// or the solver's delayed CGS2), on a block of nrhs systems stored rhs-innermost. A tile is a range of whole rows of nrhs
// elements, so the tile of basis vector i is one contiguous range of memory and
// one bulk copy per vector (plus one for w) fills a pipeline stage. The bytes in
// flight are set by the stage count and size, not by registers or occupancy.
//
// Warp 8 is the producer: its lane 0 waits until a stage is free, and its lanes
// issue the copies of the next tile into it (one vector per lane). Warps 0-7 consume: each owns whole rows of a
// tile (a lane owns EPL consecutive elements of a row, hence a fixed set of
// rhs) and ALL basis vectors for them, so
//   w'   = w - sum_i c_i v_i            (update; coefficients staged in shared memory)
//   a_i += conj(v_i) w'                 (dots, per thread and vector, in registers)
//   n   += |w'|^2                       (norm)
// need no exchange between warps: there is no block-wide barrier per tile, a warp
// releases a stage with one mbarrier arrival. (The vector-split instance for
// update + dots with 17-32 vectors and two rows per warp is the exception inside a
// warp: its two half-warps own the even / odd vectors of both rows and exchange
// partial sums by shuffles.) The per-(vector, rhs) sums over
// lanes and warps, and the norm, go to per-CTA partials in a fixed order at the
// end (deterministic, like every reduction here).
#pragma once
#include "bulk_async.cuh"
#include "kernels.h"

namespace lqcd {
namespace gss {

struct Args {
  int64_t Q;           // rows of nrhs elements (n / nrhs)
  int64_t vstride;     // elements between basis vectors
  int nrhs, nvec;
  int S;               // pipeline stages
  int TR;              // rows per tile = 8 * H * J, a multiple of 4
  int J;               // warp steps per consumer warp per tile
  int lpr, H;          // lanes per row (nrhs / EPL), rows per warp step (32 / lpr)
  int red_vecs;        // vectors per round of the final reduction
  uint32_t vt_bytes;   // bytes of one vector's tile in a stage
  uint32_t stage_bytes;
  uint32_t coef_off;   // shared-memory offsets (bytes) of the coefficients and the stages
  uint32_t stage_off;
  const void* basis;
  void* w;
  const double2* coef;
  const double* oscale;
  void* wout;
  double2* partials;
  const int* skip;
  int* err;            // set (bit 0) if a pipeline wait gave up
};

using namespace bulk;

// shared-memory loads of EPL consecutive basis elements -> FP32 complex
__device__ __forceinline__ float2 bf16pair(unsigned u) {
  return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}
template <int EPL>
__device__ __forceinline__ void lds(const float2* p, float2 (&o)[EPL]) {
  if constexpr (EPL == 2) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = make_float2(v.x, v.y);
    o[1] = make_float2(v.z, v.w);
  } else {
    o[0] = *p;
  }
}
template <int EPL>
__device__ __forceinline__ void lds(const __nv_bfloat162* p, float2 (&o)[EPL]) {
  if constexpr (EPL == 2) {
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    o[0] = bf16pair(u.x);
    o[1] = bf16pair(u.y);
  } else {
    o[0] = bf16pair(*reinterpret_cast<const unsigned*>(p));
  }
}
// global stores of the updated w: FP32 (w itself) or the basis storage type (wout)
template <int EPL>
__device__ __forceinline__ void stg(float2* p, const float2 (&v)[EPL]) {
  if constexpr (EPL == 2) *reinterpret_cast<float4*>(p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
  else *p = v[0];
}
template <int EPL>
__device__ __forceinline__ void stg(__nv_bfloat162* p, const float2 (&v)[EPL]) {
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

// acc += c v and (re, im) += conj(v) w as chains of fused multiply-adds (four per complex
// product, no separate multiply or add)
__device__ __forceinline__ void cmac(float2 c, float2 v, float2& acc) {
  acc.x = fmaf(-c.y, v.y, fmaf(c.x, v.x, acc.x));
  acc.y = fmaf(c.y, v.x, fmaf(c.x, v.y, acc.y));
}
__device__ __forceinline__ void cdot(float2 v, float2 w, float& re, float& im) {
  re = fmaf(v.y, w.y, fmaf(v.x, w.x, re));
  im = fmaf(-v.y, w.x, fmaf(v.x, w.y, im));
}

constexpr int kConsumers = 8;                 // consumer warps
constexpr int kThreads = 32 * (kConsumers + 1);

// Two CTAs per SM while the dot accumulators fit the smaller register share.
__host__ __device__ constexpr bool two_ctas(int nv, int epl) { return nv * epl <= 16; }

// NV: the largest nvec of the instance (8, 16, 24 or 32): the dot accumulators
// a_i live in registers, NV * EPL complex per thread.
// VSPLIT (dots, with or without the update; one rhs per lane, two rows per warp): the two
// half-warps split the vectors (i even / odd) instead of the rows; each handles its vectors
// for both rows of the warp, and the update's partial sums and the updated w are exchanged
// with the partner lane by one shuffle. Half the dot accumulators, room for the coefficients
// in registers, and packed FP32 (fma.rn.f32x2) for the sums.
template <typename B, int EPL, int NV, bool UPDATE, bool DOTS, bool NORM, bool VSPLIT = false>
__global__ void __launch_bounds__(kThreads, two_ctas(NV, EPL) ? 2 : 1) gs_stream_kernel(const Args a) {
  static_assert(!VSPLIT || (DOTS && EPL == 1 && NV % 2 == 0), "vector split: dots, EPL 1");
  using C = float2;
  if (a.skip != nullptr && *a.skip != 0) return;
  extern __shared__ __align__(128) unsigned char smem[];
  const int S = a.S;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + S;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + S);
  C* cs = reinterpret_cast<C*>(smem + a.coef_off);           // [nvec][nrhs] coefficients, FP32
  unsigned char* stages = smem + a.stage_off;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nrhs = a.nrhs, nvec = a.nvec, lpr = a.lpr, H = a.H, J = a.J, TR = a.TR;
  const int hrow = lane / lpr;
  const bool lane_on = hrow < H;
  const int r = (lane % lpr) * EPL;  // first rhs of this lane, the same in every row it owns
  const int64_t Q = a.Q;
  const int64_t ntiles = (Q + TR - 1) / TR;
  const int64_t G = gridDim.x;
  const int L = (int)((ntiles - blockIdx.x + G - 1) / G);  // tiles of this CTA
  const int vte = (int)(a.vt_bytes / sizeof(B));
  const B* basis = (const B*)a.basis;
  C* w = (C*)a.w;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumers);
    }
    *abort_flag = 0;
    fence_proxy_async();  // the initialised barriers are seen by the copy engine
  }
  if (UPDATE)
    for (int t = tid; t < nvec * nrhs; t += kThreads) {
      const double2 c = a.coef[t];
      cs[t] = make_float2((float)c.x, (float)c.y);
    }
  __syncthreads();

  constexpr int NA = VSPLIT ? NV / 2 : NV;  // dot accumulators per lane
  float ar[NA][EPL], ai[NA][EPL];
  float nn[EPL], sc[EPL];
#pragma unroll
  for (int q = 0; q < EPL; ++q) {
    nn[q] = 0.f;
    sc[q] = (UPDATE && a.oscale != nullptr && lane_on && warp < kConsumers) ? (float)a.oscale[r + q] : 1.f;
#pragma unroll
    for (int i = 0; i < NA; ++i) { ar[i][q] = 0.f; ai[i][q] = 0.f; }
  }

  if (warp == kConsumers) {
    // ---------------- producer: lane 0 waits for the stage and posts the byte count,
    // the lanes issue one copy each (vector i on lane i % 32, w after the vectors)
    int issued = 0;
    for (int l = 0; l < L; ++l) {
      const int s = l % S;
      const int64_t row0 = (blockIdx.x + (int64_t)l * G) * TR;
      const int64_t rows = (Q - row0) < TR ? (Q - row0) : TR;
      const uint32_t vbytes = (uint32_t)(rows * nrhs * (int64_t)sizeof(B));
      const uint32_t wbytes = (uint32_t)(rows * nrhs * (int64_t)sizeof(C));
      int go = 1;
      if (lane == 0) {
        if (l >= S && !mbar_wait_bounded(&empty[s], (uint32_t)(l / S - 1) & 1u)) {
          *abort_flag = 1;
          atomicOr(a.err, 1);
        }
        go = *abort_flag ? 0 : 1;
        if (go) mbar_expect_tx(&full[s], vbytes * (uint32_t)nvec + wbytes);
      }
      go = __shfl_sync(0xffffffffu, go, 0);
      if (!go) break;
      unsigned char* st = stages + (size_t)s * a.stage_bytes;
      for (int i = lane; i <= nvec; i += 32) {
        if (i < nvec) bulk_load(st + (size_t)i * a.vt_bytes, basis + i * a.vstride + row0 * nrhs, vbytes, &full[s]);
        else bulk_load(st + (size_t)nvec * a.vt_bytes, w + row0 * nrhs, wbytes, &full[s]);
      }
      issued = l + 1;
    }
    if (lane == 0 && *abort_flag) {
      // the copies still in flight land before the stages are reused below
      for (int l = issued - S < 0 ? 0 : issued - S; l < issued; ++l)
        mbar_wait_bounded(&full[l % S], (uint32_t)(l / S) & 1u);
    }
  } else {
    // ---------------- consumers
    // with one rhs per lane the lane's update coefficients are the same for every element
    // it visits: kept in registers (one shared-memory read per basis element fewer) where
    // the instance has the registers to spare (the 16- and 32-vector ones would spill)
    constexpr bool kCoefRegs = UPDATE && EPL == 1 && (NV == 8 || NV == 24) && !VSPLIT;
    constexpr int NC = kCoefRegs ? NA : 1;
    C cr[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k)
      cr[k] = (kCoefRegs && k < nvec && lane_on) ? cs[k * nrhs + r] : make_float2(0.f, 0.f);
    // VSPLIT works on packed FP32 pairs (fma.rn.f32x2): the coefficients of vectors 2k + hrow
    // as broadcast pairs (c.re, c.re), (c.im, c.im), and per vector the dot accumulators
    // dp = sum (v.re w.re, v.im w.im), dq = sum (v.re w.im, -v.im w.re)
    constexpr int NP = VSPLIT ? NA : 1;
    C cxx[NP], cyy[NP], dp[NP], dq[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int i = 2 * k + hrow;
      const C c = (VSPLIT && UPDATE && i < nvec && lane_on) ? cs[i * nrhs + r] : make_float2(0.f, 0.f);
      cxx[k] = make_float2(c.x, c.x);
      cyy[k] = make_float2(c.y, c.y);
      dp[k] = make_float2(0.f, 0.f);
      dq[k] = make_float2(0.f, 0.f);
    }
    // VSPLIT: the lane holding the same rhs in the other row of the warp's row pair
    const int partner = (VSPLIT && lane_on) ? (hrow == 0 ? lane + lpr : lane - lpr) : lane;
    for (int l = 0; l < L; ++l) {
      const int s = l % S;
      if (!mbar_wait_bounded(&full[s], (uint32_t)(l / S) & 1u)) {
        *abort_flag = 1;
        atomicOr(a.err, 1);
        break;
      }
      const int64_t row0 = (blockIdx.x + (int64_t)l * G) * TR;
      const int rows = (int)((Q - row0) < TR ? (Q - row0) : TR);
      const unsigned char* st = stages + (size_t)s * a.stage_bytes;
      const B* vt = reinterpret_cast<const B*>(st);
      const C* wt = reinterpret_cast<const C*>(st + (size_t)nvec * a.vt_bytes);
      if constexpr (VSPLIT) {
        for (int j = 0; j < J; ++j) {
          const int rowA = (j * kConsumers + warp) * 2;  // H == 2: the warp's rows rowA, rowA + 1
          if (rowA >= rows) continue;                     // warp-uniform
          const bool okB = rowA + 1 < rows;
          const bool mine_ok = lane_on && (hrow == 0 || okB);
          const int eA = rowA * nrhs + r, eB = eA + nrhs;
          const int e = hrow == 0 ? eA : eB;
          C wn = mine_ok ? wt[e] : make_float2(0.f, 0.f);
          if constexpr (UPDATE) {
            // partial update sums over this lane's vectors, for both rows: (sum c.re v.re, sum c.re v.im)
            // and (sum c.im v.re, sum c.im v.im) as packed pairs
            C xa = make_float2(0.f, 0.f), ya = xa, xb = xa, yb = xa;
#pragma unroll
            for (int k = 0; k < NA; ++k) {
              const int i = 2 * k + hrow;
              if (lane_on && i < nvec) {
                C va[1], vb[1] = {make_float2(0.f, 0.f)};
                lds<1>(vt + (size_t)i * vte + eA, va);
                if (okB) lds<1>(vt + (size_t)i * vte + eB, vb);
                xa = __ffma2_rn(cxx[k], va[0], xa);
                ya = __ffma2_rn(cyy[k], va[0], ya);
                xb = __ffma2_rn(cxx[k], vb[0], xb);
                yb = __ffma2_rn(cyy[k], vb[0], yb);
              }
            }
            const C pa = make_float2(xa.x - ya.y, xa.y + ya.x);
            const C pb = make_float2(xb.x - yb.y, xb.y + yb.x);
            const C mine = hrow == 0 ? pa : pb, other = hrow == 0 ? pb : pa;
            // the partner's partial for this lane's row (the partner sends its sum for the other row)
            const float ox = __shfl_sync(0xffffffffu, other.x, partner);
            const float oy = __shfl_sync(0xffffffffu, other.y, partner);
            wn = make_float2(wn.x - (mine.x + ox), wn.y - (mine.y + oy));
            if (mine_ok) {
              const C ws[1] = {make_float2(wn.x * sc[0], wn.y * sc[0])};
              if (a.wout != nullptr) stg<1>((B*)a.wout + row0 * nrhs + e, ws);
              else stg<1>(w + row0 * nrhs + e, ws);
            }
          }
          if (NORM && mine_ok) nn[0] = fmaf(wn.y, wn.y, fmaf(wn.x, wn.x, nn[0]));
          // dots of this lane's vectors with the updated w of both rows
          const float wx = __shfl_sync(0xffffffffu, wn.x, partner);
          const float wy = __shfl_sync(0xffffffffu, wn.y, partner);
          C wa = hrow == 0 ? wn : make_float2(wx, wy);
          C wb = hrow == 0 ? make_float2(wx, wy) : wn;
          if (!okB) wb = make_float2(0.f, 0.f);
          const C wa2 = make_float2(wa.y, -wa.x), wb2 = make_float2(wb.y, -wb.x);
#pragma unroll
          for (int k = 0; k < NA; ++k) {
            const int i = 2 * k + hrow;
            if (lane_on && i < nvec) {
              C va[1], vb[1] = {make_float2(0.f, 0.f)};
              lds<1>(vt + (size_t)i * vte + eA, va);
              if (okB) lds<1>(vt + (size_t)i * vte + eB, vb);
              dp[k] = __ffma2_rn(va[0], wa, dp[k]);
              dq[k] = __ffma2_rn(va[0], wa2, dq[k]);
              dp[k] = __ffma2_rn(vb[0], wb, dp[k]);
              dq[k] = __ffma2_rn(vb[0], wb2, dq[k]);
            }
          }
        }
      } else
      for (int j = 0; j < J; ++j) {
        const int row = (j * kConsumers + warp) * H + hrow;
        if (!(lane_on && row < rows)) continue;
        const int e = row * nrhs + r;
        C wn[EPL];
#pragma unroll
        for (int q = 0; q < EPL; ++q) wn[q] = wt[e + q];
        if (UPDATE) {
          // four interleaved partial sums (i mod 4), combined in a fixed order
          float pr[4][EPL], pi[4][EPL];
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < EPL; ++q) { pr[u][q] = 0.f; pi[u][q] = 0.f; }
#pragma unroll
          for (int i = 0; i < NV; ++i) {
            if (i < nvec) {
              C v[EPL];
              lds<EPL>(vt + (size_t)i * vte + e, v);
#pragma unroll
              for (int q = 0; q < EPL; ++q) {
                const C c = kCoefRegs ? cr[i < NC ? i : 0] : cs[i * nrhs + r + q];
                C acc = make_float2(pr[i & 3][q], pi[i & 3][q]);
                cmac(c, v[q], acc);
                pr[i & 3][q] = acc.x;
                pi[i & 3][q] = acc.y;
              }
            }
          }
          C ws[EPL];
#pragma unroll
          for (int q = 0; q < EPL; ++q) {
            const float sr = (pr[0][q] + pr[1][q]) + (pr[2][q] + pr[3][q]);
            const float si = (pi[0][q] + pi[1][q]) + (pi[2][q] + pi[3][q]);
            wn[q] = make_float2(wn[q].x - sr, wn[q].y - si);
            ws[q] = make_float2(wn[q].x * sc[q], wn[q].y * sc[q]);
          }
          if (a.wout != nullptr) stg<EPL>((B*)a.wout + row0 * nrhs + e, ws);
          else stg<EPL>(w + row0 * nrhs + e, ws);
        }
        if (NORM) {
#pragma unroll
          for (int q = 0; q < EPL; ++q) nn[q] = fmaf(wn[q].y, wn[q].y, fmaf(wn[q].x, wn[q].x, nn[q]));
        }
        if (DOTS) {
#pragma unroll
          for (int i = 0; i < NV; ++i) {
            if (i < nvec) {
              C v[EPL];
              lds<EPL>(vt + (size_t)i * vte + e, v);
#pragma unroll
              for (int q = 0; q < EPL; ++q) cdot(v[q], wn[q], ar[i][q], ai[i][q]);
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);  // this warp is done with the stage
      if (*abort_flag) break;
    }
    if constexpr (VSPLIT) {
#pragma unroll
      for (int k = 0; k < NA; ++k) {
        ar[k][0] = dp[k].x + dp[k].y;
        ai[k][0] = dq[k].x + dq[k].y;
      }
    }
  }

  // per-(vector, rhs) sums over the H lanes of a warp that share the rhs, then over
  // the consumer warps, in that fixed order; red_vecs vectors per round
  __syncthreads();
  double2* red = reinterpret_cast<double2*>(stages);  // [red_vecs][8 warps][EPL][32 lanes]; stages idle
  const int nslots = nvec + 1;
  const int RV = a.red_vecs;
  for (int i0 = 0; i0 < nvec; i0 += RV) {
    if (warp < kConsumers) {
#pragma unroll
      for (int i = 0; i < NV; ++i)
        if (i >= i0 && i < i0 + RV && i < nvec)
#pragma unroll
          for (int q = 0; q < EPL; ++q) {
            float vr, vi;
            if constexpr (VSPLIT) {  // vector i sits in the lanes of row group i & 1
              const bool own = (i & 1) == hrow;
              vr = own ? ar[i >> 1][q] : 0.f;
              vi = own ? ai[i >> 1][q] : 0.f;
            } else {
              vr = ar[i][q];
              vi = ai[i][q];
            }
            red[(((i - i0) * kConsumers + warp) * EPL + q) * 32 + lane] =
                make_double2(DOTS ? (double)vr : 0.0, DOTS ? (double)vi : 0.0);
          }
    }
    __syncthreads();
    for (int t2 = tid; t2 < RV * nrhs; t2 += kThreads) {
      const int di = t2 / nrhs, R = t2 % nrhs;
      const int i = i0 + di;
      if (i < nvec) {
        const int q = R % EPL, l0 = R / EPL;
        double2 acc = make_double2(0.0, 0.0);
        for (int wp = 0; wp < kConsumers; ++wp)
          for (int h = 0; h < H; ++h) {
            const double2 v = red[((di * kConsumers + wp) * EPL + q) * 32 + l0 + h * lpr];
            acc.x += v.x;
            acc.y += v.y;
          }
        a.partials[((int64_t)blockIdx.x * nslots + i) * nrhs + R] = acc;
      }
    }
    __syncthreads();
  }
  if (warp < kConsumers) {
#pragma unroll
    for (int q = 0; q < EPL; ++q) red[(warp * EPL + q) * 32 + lane] = make_double2(NORM ? (double)nn[q] : 0.0, 0.0);
  }
  __syncthreads();
  for (int R = tid; R < nrhs; R += kThreads) {
    const int q = R % EPL, l0 = R / EPL;
    double acc = 0.0;
    for (int wp = 0; wp < kConsumers; ++wp)
      for (int h = 0; h < H; ++h) acc += red[(wp * EPL + q) * 32 + l0 + h * lpr].x;
    a.partials[((int64_t)blockIdx.x * nslots + nvec) * nrhs + R] = make_double2(acc, 0.0);
  }
}

// Tile geometry for one pass; ok = false when no stage layout fits shared memory.
struct Plan {
  bool ok = false;
  int J = 1, S = 2, TR = 4, lpr = 1, H = 1, ctas_per_sm = 1, red_vecs = 1;
  uint32_t vt_bytes = 0, stage_bytes = 0, coef_off = 0, stage_off = 0;
  size_t smem = 0;
};

// nv: the instance's vector capacity (8, 16, 24 or 32)
inline Plan make_plan(int nrhs, int nvec, int nv, int epl, int elem_bytes, bool update) {
  Plan p;
  if (nrhs % epl != 0 || nrhs / epl > 32 || nvec < 1 || nvec > nv) return p;
  p.lpr = nrhs / epl;
  p.H = 32 / p.lpr;
  const int unit = kConsumers * p.H;  // rows per unit of J
  int jstep = 1;
  while ((unit * jstep) % 4 != 0) ++jstep;
  const size_t red_one = (size_t)kConsumers * epl * 32 * sizeof(double2);
  const bool two = two_ctas(nv, epl);
  const size_t budget = two ? 112 * 1024 : 225 * 1024;
  p.coef_off = 128;
  const size_t coef_bytes = update ? ((size_t)nvec * nrhs * sizeof(float2) + 127) / 128 * 128 : 0;
  p.stage_off = (uint32_t)(128 + coef_bytes);
  auto stage_of = [&](int J, uint32_t* vt) {
    const size_t TR = (size_t)unit * J;
    *vt = (uint32_t)(TR * nrhs * elem_bytes);
    const size_t stage = (size_t)nvec * *vt + TR * nrhs * sizeof(float2);
    return (stage + 127) / 128 * 128;
  };
  auto fits = [&](int J, int S) {
    uint32_t vt;
    const size_t stage = stage_of(J, &vt);
    const size_t st = (size_t)S * stage > red_one ? (size_t)S * stage : red_one;
    return p.stage_off + st <= budget;
  };
  // three stages (two where three do not fit) of the largest tile that fits: the larger
  // the tile, the larger each vector's bulk copy and the fewer copies per byte (a copy of
  // the 16-row minimum tile of a BF16 basis is only 1 KB, and the copy count, not the
  // bytes, then set the pace of the pass)
  for (int S = 3; S >= 2; --S) {
    int best = 0;
    for (int J = jstep; J <= 64; J += jstep)
      if (fits(J, S)) best = J;
    if (best > 0) {
      p.J = best;
      p.S = S;
      p.TR = unit * best;
      p.stage_bytes = (uint32_t)stage_of(best, &p.vt_bytes);
      const size_t st = (size_t)S * p.stage_bytes > red_one ? (size_t)S * p.stage_bytes : red_one;
      p.smem = p.stage_off + st;
      p.red_vecs = (int)(st / red_one);
      if (p.red_vecs > nvec) p.red_vecs = nvec;
      if (p.red_vecs < 1) p.red_vecs = 1;
      p.ctas_per_sm = two ? 2 : 1;
      p.ok = true;
      return p;
    }
  }
  return p;
}

}  // namespace gss
}  // namespace lqcd
