// C ABI: context, gauge/clover set-up, layout conversion, operator application,
// odd-even prepare/reconstruct and the Gram-Schmidt step. The solver is in solver.cu.
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>
#include <string>

#include "ctx.h"

namespace lqcd {

static thread_local std::string g_last_error;

lqcd_status set_error(lqcd_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

lqcd_status cuda_error(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation)
    return set_error(LQCD_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return set_error(LQCD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

lqcd_status workspace(lqcd_ctx ctx, const char* name, size_t bytes, void** out) {
  Buffer& b = ctx->ws[name];
  if (b.bytes < bytes) {
    if (b.p) {
      cudaError_t e = cudaFree(b.p);
      b.p = nullptr;
      b.bytes = 0;
      if (e != cudaSuccess) return cuda_error(e, "cudaFree(workspace)");
    }
    // any captured cycle graph may point at the old buffer
    if (ctx->cycle.exec) {
      cudaGraphExecDestroy(ctx->cycle.exec);
      cudaGraphDestroy(ctx->cycle.graph);
      ctx->cycle.exec = nullptr;
      ctx->cycle.graph = nullptr;
      ctx->cycle.key.clear();
    }
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
      b.p = nullptr;
      return set_error(LQCD_ERR_OOM, "workspace '%s': cannot allocate %zu bytes (%s)", name, bytes,
                       cudaGetErrorString(e));
    }
    b.bytes = bytes;
  }
  *out = b.p;
  return LQCD_OK;
}

// Device word set by the streaming kernels when a pipeline wait gives up (zeroed
// when first allocated; null if the allocation fails, which disables those kernels).
int* wait_flag(lqcd_ctx ctx) {
  const bool fresh = ctx->ws.find("wait_flag") == ctx->ws.end() || ctx->ws["wait_flag"].p == nullptr;
  void* p = nullptr;
  if (workspace(ctx, "wait_flag", sizeof(int), &p) != LQCD_OK) return nullptr;
  if (fresh && cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return nullptr;
  return (int*)p;
}

lqcd_status pinned_staging(lqcd_ctx ctx, size_t bytes, void** out) {
  if (ctx->pinned_bytes < bytes) {
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    ctx->pinned = nullptr;
    ctx->pinned_bytes = 0;
    LQCD_CUDA(cudaHostAlloc(&ctx->pinned, bytes, cudaHostAllocDefault), "cudaHostAlloc(staging)");
    ctx->pinned_bytes = bytes;
  }
  *out = ctx->pinned;
  return LQCD_OK;
}

int site_tile_log2(const lqcd_ctx_s* ctx, int nrhs) {
  int want = 0;  // S * nrhs >= 16 complex numbers per component run
  while ((1 << want) * nrhs < 16 && want < 4) ++want;
  int lim = 0;
  while (((ctx->g.Vh >> (lim + 1)) << (lim + 1)) == ctx->g.Vh && lim < want) ++lim;
  return lim < want ? lim : want;
}

PackedLayout layout_for(const lqcd_ctx_s* ctx, int nrhs) {
  PackedLayout l;
  l.nrhs = nrhs;
  l.log_s = site_tile_log2(ctx, nrhs);
  return l;
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename Real>
static DslashArgs<Real> base_args(lqcd_ctx ctx, int nrhs, bool f64) {
  DslashArgs<Real> a;
  memset(&a, 0, sizeof(a));
  a.g = ctx->g;
  a.lay = layout_for(ctx, nrhs);
  a.half_elems = (int64_t)ctx->g.Vh * 12 * nrhs;
  a.links = (const typename Cplx<Real>::T*)(f64 ? ctx->links64 : ctx->links32);
  a.blocks = (const Real*)(f64 ? ctx->blk64 : ctx->blk32);
  a.blocks_inv = (const Real*)(f64 ? ctx->inv64 : ctx->inv32);
  a.num_sms = ctx->num_sms;
  if (!f64) {
    a.links_aos = ctx->links32_aos;
    a.blocks_aos = ctx->blk32_aos;
    a.blocks_inv_aos = ctx->inv32_aos;
    a.links_r12 = ctx->links32_r12;
    a.links_r12_bf16 = ctx->links_bf16_r12;
    a.link_format = ctx->link_format == LQCD_LINKS_BF16 ? 2 : 0;
  }
  a.time_bc = (Real)ctx->time_bc;
  a.err = ctx->ws.count("wait_flag") ? (int*)ctx->ws["wait_flag"].p : nullptr;
  return a;
}

template <typename Real>
static cudaError_t run(const DslashArgs<Real>& a, int self_mode, int post_mode, int variant, cudaStream_t s) {
  return launch_dslash<Real>(a, self_mode, post_mode, variant, s);
}

template <typename Real>
static lqcd_status apply_t(lqcd_ctx ctx, int op, int nrhs, const void* in, void* out, void* tmp,
                           const int* skip, cudaStream_t stream) {
  using C = typename Cplx<Real>::T;
  const bool f64 = sizeof(Real) == 8;
  const bool clover = ctx->c_sw != 0.0;
  const Real diag = (Real)(4.0 + ctx->m0);
  const Real diag_inv = (Real)(1.0 / (4.0 + ctx->m0));
  DslashArgs<Real> a = base_args<Real>(ctx, nrhs, f64);
  a.skip = skip;
  a.hop = 1;
  const int variant = tuned_variant(ctx, f64, nrhs, op);
  if (op == LQCD_OP_FULL) {
    a.full = 1;
    a.n_target = ctx->g.V;
    a.out = (C*)out;
    a.self_in = (const C*)in;
    a.hop_in = (const C*)in;
    a.c_hop = (Real)-0.5;
    a.self_scalar = diag;
    LQCD_CUDA(run<Real>(a, clover ? SELF_BLOCK : SELF_SCALAR, POST_NONE, variant, stream), "dslash full");
    return LQCD_OK;
  }
  // Schur: pass A on even sites, t_e = A_ee^{-1} D_eo psi_o
  a.full = 0;
  a.n_target = ctx->g.Vh;
  a.target_parity = 0;
  a.out = (C*)tmp;
  a.hop_in = (const C*)in;
  a.c_hop = (Real)-0.5;
  a.post_scalar = diag_inv;
  LQCD_CUDA(run<Real>(a, SELF_NONE, clover ? POST_BLOCKINV : POST_SCALAR, variant, stream), "dslash schur A");
  // pass B on odd sites, out = A_oo psi_o - D_oe t_e
  a.target_parity = 1;
  a.out = (C*)out;
  a.hop_in = (const C*)tmp;
  a.self_in = (const C*)in;
  a.self_scalar = diag;
  a.c_hop = (Real)0.5;
  LQCD_CUDA(run<Real>(a, clover ? SELF_BLOCK : SELF_SCALAR, POST_NONE, variant, stream), "dslash schur B");
  return LQCD_OK;
}

lqcd_status apply_operator(lqcd_ctx ctx, int op, bool f64, int nrhs, const void* in, void* out,
                           void* tmp, const int* skip, cudaStream_t stream) {
  return f64 ? apply_t<double>(ctx, op, nrhs, in, out, tmp, skip, stream)
             : apply_t<float>(ctx, op, nrhs, in, out, tmp, skip, stream);
}

// The operator on a BF16-stored input block with FP32 arithmetic, FP32 output
// (and FP32 Schur intermediate tmp).
lqcd_status apply_operator_bf16in(lqcd_ctx ctx, int op, int nrhs, const void* in, void* out, void* tmp,
                                  const int* skip, cudaStream_t stream) {
  const bool clover = ctx->c_sw != 0.0;
  DslashArgs<float> a = base_args<float>(ctx, nrhs, false);
  a.skip = skip;
  a.hop = 1;
  if (op == LQCD_OP_FULL) {
    a.full = 1;
    a.n_target = ctx->g.V;
    a.out = (float2*)out;
    a.self_in = (const float2*)in;   // BF16 storage, reinterpreted by the kernel
    a.hop_in = (const float2*)in;
    a.c_hop = -0.5f;
    a.self_scalar = (float)(4.0 + ctx->m0);
    LQCD_CUDA(launch_dslash_bf16(a, clover ? SELF_BLOCK : SELF_SCALAR, POST_NONE, true, stream), "dslash bf16 full");
    return LQCD_OK;
  }
  a.full = 0;
  a.n_target = ctx->g.Vh;
  a.target_parity = 0;
  a.out = (float2*)tmp;
  a.hop_in = (const float2*)in;
  a.c_hop = -0.5f;
  a.post_scalar = (float)(1.0 / (4.0 + ctx->m0));
  LQCD_CUDA(launch_dslash_bf16(a, SELF_NONE, clover ? POST_BLOCKINV : POST_SCALAR, true, stream), "dslash bf16 A");
  a.target_parity = 1;
  a.out = (float2*)out;
  a.hop_in = (const float2*)tmp;
  a.self_in = (const float2*)in;
  a.self_scalar = (float)(4.0 + ctx->m0);
  a.c_hop = 0.5f;
  LQCD_CUDA(launch_dslash_bf16(a, clover ? SELF_BLOCK : SELF_SCALAR, POST_NONE, false, stream), "dslash bf16 B");
  return LQCD_OK;
}

template <typename Real>
static lqcd_status prepare_t(lqcd_ctx ctx, int nrhs, const void* b_full, void* bhat_o, void* tmp_even,
                             cudaStream_t stream) {
  using C = typename Cplx<Real>::T;
  const bool clover = ctx->c_sw != 0.0;
  DslashArgs<Real> a = base_args<Real>(ctx, nrhs, sizeof(Real) == 8);
  const C* b = (const C*)b_full;
  // u_e = A_ee^{-1} b_e (site-local)
  a.full = 0;
  a.n_target = ctx->g.Vh;
  a.target_parity = 0;
  a.hop = 0;
  a.out = (C*)tmp_even;
  a.self_in = b;
  a.self_scalar = (Real)1;
  a.post_scalar = (Real)(1.0 / (4.0 + ctx->m0));
  LQCD_CUDA(run<Real>(a, SELF_SCALAR, clover ? POST_BLOCKINV : POST_SCALAR, -1, stream), "prepare A_ee^-1");
  // hat b_o = b_o - D_oe u_e = b_o + (1/2) H u_e
  a.target_parity = 1;
  a.hop = 1;
  a.out = (C*)bhat_o;
  a.self_in = b + a.half_elems;
  a.hop_in = (const C*)tmp_even;
  a.c_hop = (Real)0.5;
  LQCD_CUDA(run<Real>(a, SELF_SCALAR, POST_NONE, -1, stream), "prepare hop");
  return LQCD_OK;
}

template <typename Real>
static lqcd_status reconstruct_t(lqcd_ctx ctx, int nrhs, const void* b_full, const void* x_o,
                                 void* x_full, cudaStream_t stream) {
  using C = typename Cplx<Real>::T;
  const bool clover = ctx->c_sw != 0.0;
  DslashArgs<Real> a = base_args<Real>(ctx, nrhs, sizeof(Real) == 8);
  // x_e = A_ee^{-1} (b_e - D_eo x_o) = A_ee^{-1} (b_e + (1/2) H x_o)
  a.full = 0;
  a.n_target = ctx->g.Vh;
  a.target_parity = 0;
  a.hop = 1;
  a.out = (C*)x_full;
  a.self_in = (const C*)b_full;
  a.self_scalar = (Real)1;
  a.hop_in = (const C*)x_o;
  a.c_hop = (Real)0.5;
  a.post_scalar = (Real)(1.0 / (4.0 + ctx->m0));
  LQCD_CUDA(run<Real>(a, SELF_SCALAR, clover ? POST_BLOCKINV : POST_SCALAR, -1, stream), "reconstruct");
  C* xo_dst = (C*)x_full + a.half_elems;
  if ((const void*)xo_dst != x_o)
    LQCD_CUDA(cudaMemcpyAsync(xo_dst, x_o, sizeof(C) * a.half_elems, cudaMemcpyDeviceToDevice, stream),
              "reconstruct copy x_o");
  return LQCD_OK;
}

lqcd_status schur_prepare(lqcd_ctx ctx, bool f64, int nrhs, const void* b_full, void* bhat_o,
                          void* tmp_even, cudaStream_t stream) {
  return f64 ? prepare_t<double>(ctx, nrhs, b_full, bhat_o, tmp_even, stream)
             : prepare_t<float>(ctx, nrhs, b_full, bhat_o, tmp_even, stream);
}

lqcd_status schur_reconstruct(lqcd_ctx ctx, bool f64, int nrhs, const void* b_full, const void* x_o,
                              void* x_full, cudaStream_t stream) {
  return f64 ? reconstruct_t<double>(ctx, nrhs, b_full, x_o, x_full, stream)
             : reconstruct_t<float>(ctx, nrhs, b_full, x_o, x_full, stream);
}

}  // namespace lqcd

using namespace lqcd;

// ------------------------------------------------------------------ C ABI

#define CHECK_CTX(ctx) \
  if ((ctx) == nullptr) return set_error(LQCD_ERR_ARG, "%s: null context", __func__)

static lqcd_status check_ready(lqcd_ctx ctx, const char* fn) {
  if (!ctx->have_gauge) return set_error(LQCD_ERR_STATE, "%s: lqcd_set_gauge has not been called", fn);
  if (!ctx->have_blocks) return set_error(LQCD_ERR_STATE, "%s: lqcd_set_clover has not been called", fn);
  return LQCD_OK;
}

static bool valid_dtype(int d) { return d == LQCD_C64 || d == LQCD_C128; }
static bool valid_storage(int d) { return d == LQCD_C64 || d == LQCD_C128 || d == LQCD_BF16S; }
static size_t elem_bytes(int d) { return d == LQCD_C128 ? 16 : (d == LQCD_C64 ? 8 : 4); }
static bool valid_sites(int s) { return s == LQCD_SITES_FULL || s == LQCD_SITES_EVEN || s == LQCD_SITES_ODD; }

extern "C" {

const char* lqcd_status_string(lqcd_status s) {
  switch (s) {
    case LQCD_OK: return "ok";
    case LQCD_NOT_CONVERGED: return "not converged";
    case LQCD_ERR_ARG: return "invalid argument";
    case LQCD_ERR_OOM: return "out of memory";
    case LQCD_ERR_CUDA: return "CUDA error";
    case LQCD_ERR_NONFINITE: return "non-finite value";
    case LQCD_ERR_SINGULAR: return "singular site block";
    case LQCD_ERR_STATE: return "call out of order";
    default: return "unknown status";
  }
}

const char* lqcd_last_error(void) { return g_last_error.c_str(); }

lqcd_status lqcd_create(const int dims[4], int time_bc, lqcd_ctx* out) {
  if (out == nullptr || dims == nullptr) return set_error(LQCD_ERR_ARG, "lqcd_create: null pointer");
  *out = nullptr;
  long long V = 1;
  for (int k = 0; k < 4; ++k) {
    if (dims[k] < 2 || dims[k] % 2 != 0)
      return set_error(LQCD_ERR_ARG, "lqcd_create: extent %d of direction %d is not even and >= 2",
                       dims[k], k);
    V *= dims[k];
  }
  if (V * 12 > (1LL << 31))
    return set_error(LQCD_ERR_ARG, "lqcd_create: %lld sites exceed the 2^31/12 limit", V);
  if (time_bc != 1 && time_bc != -1)
    return set_error(LQCD_ERR_ARG, "lqcd_create: time_bc must be +1 or -1, got %d", time_bc);
  lqcd_ctx c = new (std::nothrow) lqcd_ctx_s();
  if (!c) return set_error(LQCD_ERR_OOM, "lqcd_create: host allocation failed");
  for (int k = 0; k < 4; ++k) c->dims[k] = dims[k];
  c->g = make_geom(dims);
  c->time_bc = time_bc;
  *out = c;
  return LQCD_OK;
}

static void free_ptr(void*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

lqcd_status lqcd_free(lqcd_ctx ctx) {
  if (!ctx) return LQCD_OK;
  cudaDeviceSynchronize();
  if (ctx->cycle.exec) cudaGraphExecDestroy(ctx->cycle.exec);
  if (ctx->cycle.graph) cudaGraphDestroy(ctx->cycle.graph);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  for (auto& e : ctx->prof_events) cudaEventDestroy(e);
  free_ptr(ctx->links64); free_ptr(ctx->links32);
  free_ptr(ctx->blk64); free_ptr(ctx->inv64); free_ptr(ctx->blk32); free_ptr(ctx->inv32);
  free_ptr(ctx->links32_aos); free_ptr(ctx->blk32_aos); free_ptr(ctx->inv32_aos);
  free_ptr(ctx->links32_r12); free_ptr(ctx->links_bf16_r12);
  void* e = ctx->d_err; free_ptr(e);
  for (auto& kv : ctx->ws) free_ptr(kv.second.p);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  delete ctx;
  return LQCD_OK;
}

lqcd_status lqcd_set_gauge(lqcd_ctx ctx, const void* U, void* stream) {
  CHECK_CTX(ctx);
  if (!U) return set_error(LQCD_ERR_ARG, "lqcd_set_gauge: null gauge field");
  cudaStream_t s = (cudaStream_t)stream;
  LQCD_CUDA(cudaGetDevice(&ctx->device), "cudaGetDevice");
  LQCD_CUDA(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device),
            "cudaDeviceGetAttribute");
  const size_t V = ctx->g.V;
  if (!ctx->links64) {
    LQCD_CUDA(cudaMalloc(&ctx->links64, 36 * V * sizeof(double2)), "cudaMalloc(links64)");
    LQCD_CUDA(cudaMalloc(&ctx->links32, 36 * V * sizeof(float2)), "cudaMalloc(links32)");
    LQCD_CUDA(cudaMalloc((void**)&ctx->d_err, sizeof(int)), "cudaMalloc(err)");
    LQCD_CUDA(cudaMalloc(&ctx->links32_aos, 40 * V * sizeof(float2)), "cudaMalloc(links32 site-major)");
    LQCD_CUDA(cudaMalloc(&ctx->links32_r12, 24 * V * sizeof(float2)), "cudaMalloc(links32 two rows)");
    LQCD_CUDA(cudaMalloc(&ctx->links_bf16_r12, 24 * V * sizeof(__nv_bfloat162)), "cudaMalloc(links bf16 two rows)");
    if (wait_flag(ctx) == nullptr) return set_error(LQCD_ERR_OOM, "lqcd_set_gauge: cannot allocate the wait flag");
  }
  const void* src = U;
  if (!is_device_pointer(U)) {
    void* tmp;
    lqcd_status st = workspace(ctx, "gauge_upload", 36 * V * sizeof(double2), &tmp);
    if (st != LQCD_OK) return st;
    LQCD_CUDA(cudaMemcpyAsync(tmp, U, 36 * V * sizeof(double2), cudaMemcpyHostToDevice, s),
              "upload gauge field");
    src = tmp;
  }
  LQCD_CUDA(launch_gauge_pack(ctx->g, ctx->time_bc, src, ctx->links64, ctx->links32, s), "gauge pack");
  LQCD_CUDA(launch_links_aos(ctx->g.V, ctx->links32, ctx->links32_aos, s), "links site-major");
  LQCD_CUDA(launch_links_r12(ctx->g.V, ctx->links32, ctx->links32_r12, ctx->links_bf16_r12, s), "links two rows");
  if (src != U) LQCD_CUDA(cudaStreamSynchronize(s), "gauge upload sync");
  ctx->have_gauge = true;
  ctx->have_blocks = false;
  return LQCD_OK;
}

lqcd_status lqcd_set_clover(lqcd_ctx ctx, double m0, double c_sw, void* stream) {
  CHECK_CTX(ctx);
  if (!ctx->have_gauge) return set_error(LQCD_ERR_STATE, "lqcd_set_clover: lqcd_set_gauge has not been called");
  if (!(4.0 + m0 != 0.0) || m0 != m0 || c_sw != c_sw)
    return set_error(LQCD_ERR_ARG, "lqcd_set_clover: invalid m0 %g or c_sw %g", m0, c_sw);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t V = ctx->g.V;
  if (!ctx->blk64) {
    LQCD_CUDA(cudaMalloc(&ctx->blk64, 72 * V * sizeof(double)), "cudaMalloc(blocks64)");
    LQCD_CUDA(cudaMalloc(&ctx->inv64, 72 * V * sizeof(double)), "cudaMalloc(inv64)");
    LQCD_CUDA(cudaMalloc(&ctx->blk32, 72 * V * sizeof(float)), "cudaMalloc(blocks32)");
    LQCD_CUDA(cudaMalloc(&ctx->inv32, 72 * V * sizeof(float)), "cudaMalloc(inv32)");
    LQCD_CUDA(cudaMalloc(&ctx->blk32_aos, 72 * V * sizeof(float)), "cudaMalloc(blocks32 site-major)");
    LQCD_CUDA(cudaMalloc(&ctx->inv32_aos, 72 * V * sizeof(float)), "cudaMalloc(inv32 site-major)");
  }
  void* leaf;
  lqcd_status st = workspace(ctx, "clover_leaves", 54 * V * sizeof(double2), &leaf);
  if (st != LQCD_OK) return st;
  LQCD_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), s), "memset err");
  LQCD_CUDA(launch_clover_build(ctx->g, ctx->links64, m0, c_sw, leaf, ctx->blk64, ctx->inv64, ctx->blk32,
                                ctx->inv32, ctx->d_err, s),
            "clover build");
  LQCD_CUDA(launch_blocks_aos(ctx->g.V, ctx->blk32, ctx->blk32_aos, s), "blocks site-major");
  LQCD_CUDA(launch_blocks_aos(ctx->g.V, ctx->inv32, ctx->inv32_aos, s), "inverse blocks site-major");
  int herr = 0;
  LQCD_CUDA(cudaMemcpyAsync(&herr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, s), "read err");
  LQCD_CUDA(cudaStreamSynchronize(s), "clover sync");
  ctx->m0 = m0;
  ctx->c_sw = c_sw;
  if (herr & DEV_ERR_SINGULAR) {
    ctx->have_blocks = false;
    return set_error(LQCD_ERR_SINGULAR, "lqcd_set_clover: a 6x6 site block of A = (4+m0) - C is singular");
  }
  ctx->have_blocks = true;
  return LQCD_OK;
}

lqcd_status lqcd_export_blocks(lqcd_ctx ctx, int which, void* out, void* stream) {
  CHECK_CTX(ctx);
  lqcd_status st = check_ready(ctx, "lqcd_export_blocks");
  if (st != LQCD_OK) return st;
  if (!out || (which != 0 && which != 1)) return set_error(LQCD_ERR_ARG, "lqcd_export_blocks: bad arguments");
  LQCD_CUDA(launch_blocks_export(ctx->g, which == 0 ? ctx->blk64 : ctx->inv64, out, (cudaStream_t)stream),
            "export blocks");
  return LQCD_OK;
}

int lqcd_site_tile(lqcd_ctx ctx, int nrhs) {
  if (!ctx || nrhs < 1) return 0;
  return 1 << site_tile_log2(ctx, nrhs);
}

size_t lqcd_packed_bytes(lqcd_ctx ctx, lqcd_dtype dtype, lqcd_sites sites, int nrhs) {
  if (!ctx || !valid_storage(dtype) || !valid_sites(sites) || nrhs < 1) return 0;
  return packed_elems(ctx, sites, nrhs) * elem_bytes(dtype);
}

static lqcd_status layout_common(lqcd_ctx ctx, lqcd_dtype dtype, lqcd_sites sites, int nrhs,
                                 const void* in, void* out, void* stream, bool to_packed, const char* fn) {
  CHECK_CTX(ctx);
  if (!valid_storage(dtype) || !valid_sites(sites) || nrhs < 1 || nrhs > 256 || !in || !out)
    return set_error(LQCD_ERR_ARG, "%s: bad arguments", fn);
  const int sites_code = sites == LQCD_SITES_FULL ? 0 : 1;
  LQCD_CUDA(launch_spinor_layout(ctx->g, sites_code, nrhs, site_tile_log2(ctx, nrhs), to_packed,
                                 dtype == LQCD_C128, in, out, (cudaStream_t)stream, dtype == LQCD_BF16S),
            fn);
  return LQCD_OK;
}

lqcd_status lqcd_pack(lqcd_ctx ctx, lqcd_dtype dtype, lqcd_sites sites, int nrhs, const void* in, void* out,
                      void* stream) {
  return layout_common(ctx, dtype, sites, nrhs, in, out, stream, true, "lqcd_pack");
}

lqcd_status lqcd_unpack(lqcd_ctx ctx, lqcd_dtype dtype, lqcd_sites sites, int nrhs, const void* in,
                        void* out, void* stream) {
  return layout_common(ctx, dtype, sites, nrhs, in, out, stream, false, "lqcd_unpack");
}

lqcd_status lqcd_apply_packed(lqcd_ctx ctx, lqcd_op op, lqcd_dtype dtype, int nrhs, const void* in,
                              void* out, void* stream) {
  CHECK_CTX(ctx);
  lqcd_status st = check_ready(ctx, "lqcd_apply_packed");
  if (st != LQCD_OK) return st;
  if ((op != LQCD_OP_FULL && op != LQCD_OP_SCHUR) || !valid_storage(dtype) || nrhs < 1 || nrhs > 256 || !in ||
      !out || in == out || (dtype == LQCD_BF16S && nrhs > 128))
    return set_error(LQCD_ERR_ARG, "lqcd_apply_packed: bad arguments");
  void* tmp = nullptr;
  const lqcd_dtype tmp_type = dtype == LQCD_C128 ? LQCD_C128 : LQCD_C64;
  if (op == LQCD_OP_SCHUR) {
    st = workspace(ctx, dtype == LQCD_C128 ? "schur_tmp64" : "schur_tmp32",
                   lqcd_packed_bytes(ctx, tmp_type, LQCD_SITES_EVEN, nrhs), &tmp);
    if (st != LQCD_OK) return st;
  }
  if (dtype == LQCD_BF16S)
    return apply_operator_bf16in(ctx, op, nrhs, in, out, tmp, nullptr, (cudaStream_t)stream);
  return apply_operator(ctx, op, dtype == LQCD_C128, nrhs, in, out, tmp, nullptr, (cudaStream_t)stream);
}

lqcd_status lqcd_apply(lqcd_ctx ctx, lqcd_op op, lqcd_dtype dtype, int nrhs, const void* in, void* out,
                       void* stream) {
  CHECK_CTX(ctx);
  lqcd_status st = check_ready(ctx, "lqcd_apply");
  if (st != LQCD_OK) return st;
  if ((op != LQCD_OP_FULL && op != LQCD_OP_SCHUR) || !valid_storage(dtype) || nrhs < 1 || nrhs > 256 || !in ||
      !out)
    return set_error(LQCD_ERR_ARG, "lqcd_apply: bad arguments");
  const lqcd_sites sites = op == LQCD_OP_FULL ? LQCD_SITES_FULL : LQCD_SITES_ODD;
  const lqcd_dtype out_type = dtype == LQCD_BF16S ? LQCD_C64 : dtype;   // BF16 input gives a complex64 result
  void *pin, *pout;
  st = workspace(ctx, "apply_in", lqcd_packed_bytes(ctx, dtype, sites, nrhs), &pin);
  if (st != LQCD_OK) return st;
  st = workspace(ctx, "apply_out", lqcd_packed_bytes(ctx, out_type, sites, nrhs), &pout);
  if (st != LQCD_OK) return st;
  st = lqcd_pack(ctx, dtype, sites, nrhs, in, pin, stream);
  if (st != LQCD_OK) return st;
  st = lqcd_apply_packed(ctx, op, dtype, nrhs, pin, pout, stream);
  if (st != LQCD_OK) return st;
  return lqcd_unpack(ctx, out_type, sites, nrhs, pout, out, stream);
}

lqcd_status lqcd_schur_prepare(lqcd_ctx ctx, lqcd_dtype dtype, int nrhs, const void* b, void* bhat_o,
                               void* stream) {
  CHECK_CTX(ctx);
  lqcd_status st = check_ready(ctx, "lqcd_schur_prepare");
  if (st != LQCD_OK) return st;
  if (!valid_dtype(dtype) || nrhs < 1 || nrhs > 256 || !b || !bhat_o)
    return set_error(LQCD_ERR_ARG, "lqcd_schur_prepare: bad arguments");
  void* tmp;
  st = workspace(ctx, dtype == LQCD_C128 ? "schur_tmp64" : "schur_tmp32",
                 lqcd_packed_bytes(ctx, dtype, LQCD_SITES_EVEN, nrhs), &tmp);
  if (st != LQCD_OK) return st;
  return schur_prepare(ctx, dtype == LQCD_C128, nrhs, b, bhat_o, tmp, (cudaStream_t)stream);
}

lqcd_status lqcd_schur_reconstruct(lqcd_ctx ctx, lqcd_dtype dtype, int nrhs, const void* b, const void* x_o,
                                   void* x, void* stream) {
  CHECK_CTX(ctx);
  lqcd_status st = check_ready(ctx, "lqcd_schur_reconstruct");
  if (st != LQCD_OK) return st;
  if (!valid_dtype(dtype) || nrhs < 1 || nrhs > 256 || !b || !x_o || !x)
    return set_error(LQCD_ERR_ARG, "lqcd_schur_reconstruct: bad arguments");
  return schur_reconstruct(ctx, dtype == LQCD_C128, nrhs, b, x_o, x, (cudaStream_t)stream);
}


lqcd_status lqcd_set_kernel_variant(lqcd_ctx ctx, lqcd_dtype dtype, int nrhs, lqcd_op op, int variant) {
  CHECK_CTX(ctx);
  const bool f64 = dtype == LQCD_C128;
  if (!valid_dtype(dtype) || nrhs < 1 || nrhs > 256 || (op != LQCD_OP_FULL && op != LQCD_OP_SCHUR) ||
      (variant != -1 && !dslash_variant_ok(f64, variant, nrhs)))
    return set_error(LQCD_ERR_ARG, "lqcd_set_kernel_variant: bad arguments or variant %d does not fit nrhs %d",
                     variant, nrhs);
  if (variant == -1) ctx->tuned.erase(tune_key(f64, nrhs, op));
  else ctx->tuned[tune_key(f64, nrhs, op)] = variant;
  return LQCD_OK;
}

int lqcd_get_kernel_variant(lqcd_ctx ctx, lqcd_dtype dtype, int nrhs, lqcd_op op) {
  if (!ctx || !valid_dtype(dtype) || nrhs < 1) return -2;
  const bool f64 = dtype == LQCD_C128;
  const int v = tuned_variant(ctx, f64, nrhs, op);
  return v >= 0 ? v : dslash_default_variant(f64, nrhs);
}

int lqcd_kernel_variant_count(lqcd_dtype dtype) {
  if (!valid_dtype(dtype)) return 0;
  return dslash_variant_count(dtype == LQCD_C128);
}

lqcd_status lqcd_set_link_storage(lqcd_ctx ctx, int format) {
  CHECK_CTX(ctx);
  if (format != LQCD_LINKS_FP32 && format != LQCD_LINKS_BF16)
    return set_error(LQCD_ERR_ARG, "lqcd_set_link_storage: unknown format %d", format);
  ctx->link_format = format;
  if (ctx->cycle.exec) {  // a captured solver cycle holds the previous kernels
    cudaGraphExecDestroy(ctx->cycle.exec);
    cudaGraphDestroy(ctx->cycle.graph);
    ctx->cycle.exec = nullptr;
    ctx->cycle.graph = nullptr;
    ctx->cycle.key.clear();
  }
  return LQCD_OK;
}

int lqcd_get_link_storage(lqcd_ctx ctx) { return ctx ? ctx->link_format : -1; }

int lqcd_kernel_variant_link_reals(lqcd_dtype dtype, int variant) {
  if (!valid_dtype(dtype) || variant < 0 || variant >= dslash_variant_count(dtype == LQCD_C128)) return -1;
  return dslash_variant(dtype == LQCD_C128, variant).links == 1 ? 12 : 18;
}

lqcd_status lqcd_kernel_variant_shape(lqcd_dtype dtype, int variant, int* shape) {
  if (!valid_dtype(dtype) || shape == nullptr || variant < 0 || variant >= dslash_variant_count(dtype == LQCD_C128))
    return set_error(LQCD_ERR_ARG, "lqcd_kernel_variant_shape: bad dtype, variant or null shape");
  const DslashVariant v = dslash_variant(dtype == LQCD_C128, variant);
  const int f[11] = {v.nr, v.threads, v.minb, v.stages, v.nrhs_fixed, v.prefetch, v.ring_warps, v.ring_slots,
                     v.links == 1 ? 12 : 18, v.order, v.pipe};
  for (int i = 0; i < 11; ++i) shape[i] = f[i];
  return LQCD_OK;
}

lqcd_status lqcd_tune(lqcd_ctx ctx, lqcd_dtype dtype, int nrhs, int reps, double* times_ms, int* n_variants,
                      void* stream) {
  CHECK_CTX(ctx);
  lqcd_status st = check_ready(ctx, "lqcd_tune");
  if (st != LQCD_OK) return st;
  if (!valid_dtype(dtype) || nrhs < 1 || nrhs > 256 || reps < 1)
    return set_error(LQCD_ERR_ARG, "lqcd_tune: bad arguments");
  const bool f64 = dtype == LQCD_C128;
  cudaStream_t s = (cudaStream_t)stream;
  const int nv = dslash_variant_count(f64);
  if (n_variants) *n_variants = nv;
  const size_t full_b = lqcd_packed_bytes(ctx, dtype, LQCD_SITES_FULL, nrhs);
  void *in, *out, *tmp;
  if ((st = workspace(ctx, "tune_in", full_b, &in)) != LQCD_OK) return st;
  if ((st = workspace(ctx, "tune_out", full_b, &out)) != LQCD_OK) return st;
  if ((st = workspace(ctx, "tune_tmp", full_b / 2, &tmp)) != LQCD_OK) return st;
  LQCD_CUDA(cudaMemsetAsync(in, 0x3c, full_b, s), "tune fill");
  cudaEvent_t e0, e1;
  LQCD_CUDA(cudaEventCreate(&e0), "event");
  LQCD_CUDA(cudaEventCreate(&e1), "event");
  const int ops[2] = {LQCD_OP_FULL, LQCD_OP_SCHUR};
  for (int oi = 0; oi < 2; ++oi) {
    const int op = ops[oi];
    double best = 1e300;
    int best_v = -1;
    ctx->tuned.erase(tune_key(f64, nrhs, op));
    for (int v = 0; v < nv; ++v) {
      double med = NAN;
      if (dslash_variant_ok(f64, v, nrhs)) {
        ctx->tuned[tune_key(f64, nrhs, op)] = v;
        std::vector<float> t(reps);
        for (int w = 0; w < 2; ++w)
          if ((st = apply_operator(ctx, op, f64, nrhs, in, out, tmp, nullptr, s)) != LQCD_OK) break;
        for (int k = 0; k < reps && st == LQCD_OK; ++k) {
          cudaEventRecord(e0, s);
          st = apply_operator(ctx, op, f64, nrhs, in, out, tmp, nullptr, s);
          cudaEventRecord(e1, s);
          cudaEventSynchronize(e1);
          cudaEventElapsedTime(&t[k], e0, e1);
        }
        if (st != LQCD_OK) break;
        std::sort(t.begin(), t.end());
        med = t[reps / 2];
        if (med < best) { best = med; best_v = v; }
      }
      if (times_ms) times_ms[2 * v + oi] = med;
    }
    if (st != LQCD_OK) {
      ctx->tuned.erase(tune_key(f64, nrhs, op));
      break;
    }
    ctx->tuned[tune_key(f64, nrhs, op)] = best_v;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

}  // extern "C"
