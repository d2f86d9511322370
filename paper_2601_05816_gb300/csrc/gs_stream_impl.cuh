// Host dispatch of the streaming Gram-Schmidt kernel for one basis storage type
// (included once per storage type, so the instances compile in parallel).
#pragma once
#include "gs_stream.cuh"

namespace lqcd {
namespace gss {

template <typename B, int EPL, int NV, bool U, bool D, bool N, bool VS = false>
static cudaError_t launch_one(const Plan& p, int blocks, const Args& a, cudaStream_t s) {
  auto k = gs_stream_kernel<B, EPL, NV, U, D, N, VS>;
  // allow the largest layout make_plan can choose, once per device
  static unsigned configured = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 32 && !(configured & (1u << dev))) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 225 * 1024);
    if (e != cudaSuccess) return e;
    configured |= 1u << dev;
  } else if (dev >= 32 && p.smem > 48 * 1024) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return e;
  }
  k<<<blocks, kThreads, p.smem, s>>>(a);
  return cudaGetLastError();
}

template <typename B, int EPL, int NV>
static cudaError_t launch_flags(bool up, bool dots, bool norm, const Plan& p, int blocks, const Args& a,
                                cudaStream_t s) {
  // dots (with or without the update) with two rows per warp and 17-32 vectors: the
  // vector-split consumers
  if constexpr (EPL == 1 && NV >= 24) {
    if (up && dots && p.H == 2) {
      if (norm) return launch_one<B, EPL, NV, true, true, true, true>(p, blocks, a, s);
      return launch_one<B, EPL, NV, true, true, false, true>(p, blocks, a, s);
    }
    if (!up && dots && norm && p.H == 2) return launch_one<B, EPL, NV, false, true, true, true>(p, blocks, a, s);
  }
  if (up && dots && norm) return launch_one<B, EPL, NV, true, true, true>(p, blocks, a, s);
  if (!up && dots && norm) return launch_one<B, EPL, NV, false, true, true>(p, blocks, a, s);
  if (up && dots) return launch_one<B, EPL, NV, true, true, false>(p, blocks, a, s);
  if (up && norm) return launch_one<B, EPL, NV, true, false, true>(p, blocks, a, s);
  if (up) return launch_one<B, EPL, NV, true, false, false>(p, blocks, a, s);
  if (dots && !norm) return launch_one<B, EPL, NV, false, true, false>(p, blocks, a, s);
  return cudaErrorNotSupported;
}

template <typename B>
static cudaError_t launch_stream(const BlasPlan& plan, int64_t n, int nvec, const void* basis, int64_t vstride,
                                 void* w, const void* coef, bool update, bool dots, bool norm, void* partials,
                                 const int* skip, cudaStream_t stream, const double* oscale, void* wout,
                                 int* blocks_used) {
  const int nrhs = plan.nrhs;
  const int epl = nrhs <= 32 ? 1 : 2;
  if (plan.wait_flag == nullptr || nrhs > 64 || (nrhs > 32 && nrhs % 2 != 0) || n % nrhs != 0)
    return cudaErrorNotSupported;
  if (!(update || dots)) return cudaErrorNotSupported;
  // bulk copies: 16-byte aligned sources and sizes
  if (((uintptr_t)basis & 15) || ((uintptr_t)w & 15) || ((vstride * (int64_t)sizeof(B)) & 15) ||
      ((n * (int64_t)sizeof(B)) & 15))
    return cudaErrorNotSupported;
  if (nvec > 32) return cudaErrorNotSupported;
  const int nv = nvec <= 8 ? 8 : (nvec <= 16 ? 16 : (nvec <= 24 ? 24 : 32));
  const Plan p = make_plan(nrhs, nvec, nv, epl, (int)sizeof(B), update);
  if (!p.ok) return cudaErrorNotSupported;
  Args a;
  a.Q = n / nrhs;
  a.vstride = vstride;
  a.nrhs = nrhs;
  a.nvec = nvec;
  a.S = p.S;
  a.TR = p.TR;
  a.J = p.J;
  a.lpr = p.lpr;
  a.H = p.H;
  a.red_vecs = p.red_vecs;
  a.vt_bytes = p.vt_bytes;
  a.stage_bytes = p.stage_bytes;
  a.coef_off = p.coef_off;
  a.stage_off = p.stage_off;
  a.basis = basis;
  a.w = w;
  a.coef = (const double2*)coef;
  a.oscale = oscale;
  a.wout = wout;
  a.partials = (double2*)partials;
  a.skip = skip;
  a.err = plan.wait_flag;
  const int64_t ntiles = (a.Q + p.TR - 1) / p.TR;
  int64_t blocks = (int64_t)p.ctas_per_sm * plan.num_sms;
  if (blocks > plan.blocks) blocks = plan.blocks;  // the partials buffer holds plan.blocks CTAs
  if (blocks > ntiles) blocks = ntiles;
  if (blocks < 1) blocks = 1;
  *blocks_used = (int)blocks;
#define GSS_NV(E)                                                                                   \
  if (nv == 8) return launch_flags<B, E, 8>(update, dots, norm, p, (int)blocks, a, stream);         \
  if (nv == 16) return launch_flags<B, E, 16>(update, dots, norm, p, (int)blocks, a, stream);       \
  if (nv == 24) return launch_flags<B, E, 24>(update, dots, norm, p, (int)blocks, a, stream);       \
  return launch_flags<B, E, 32>(update, dots, norm, p, (int)blocks, a, stream);
  if (epl == 1) {
    GSS_NV(1)
  } else {
    GSS_NV(2)
  }
#undef GSS_NV
}

// Whether launch_stream runs the dot + norm pass and the update + dot + norm pass for
// every basis size up to nvec_max on this plan and vector length.
template <typename B>
static bool passes_supported(const BlasPlan& plan, int64_t n, int nvec_max) {
  const int nrhs = plan.nrhs;
  if (plan.wait_flag == nullptr || nrhs > 64 || (nrhs > 32 && nrhs % 2 != 0) || n % nrhs != 0) return false;
  if (((n * (int64_t)sizeof(B)) & 15) || nvec_max > 32 || nvec_max < 1) return false;
  const int epl = nrhs <= 32 ? 1 : 2;
  for (int nvec = 1; nvec <= nvec_max; ++nvec) {
    const int nv = nvec <= 8 ? 8 : (nvec <= 16 ? 16 : (nvec <= 24 ? 24 : 32));
    if (!make_plan(nrhs, nvec, nv, epl, (int)sizeof(B), false).ok) return false;
    if (!make_plan(nrhs, nvec, nv, epl, (int)sizeof(B), true).ok) return false;
  }
  return true;
}

}  // namespace gss
}  // namespace lqcd
