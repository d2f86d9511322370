// Library context and host-side helpers shared by the C ABI translation units.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/lqcd.h"
#include "dslash.cuh"
#include "kernels.h"

namespace lqcd {

struct Buffer {
  void* p = nullptr;
  size_t bytes = 0;
};

struct CycleGraph {
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  std::string key;
};

}  // namespace lqcd

struct lqcd_ctx_s {
  lqcd::Geom g;
  int dims[4];
  int time_bc = -1;
  int num_sms = 152;
  int device = 0;
  bool have_gauge = false;
  bool have_blocks = false;
  double m0 = 0.0, c_sw = 0.0;
  void* links64 = nullptr;  // [4][9][V] double2
  void* links32 = nullptr;  // [4][9][V] float2
  void* blk64 = nullptr;    // A, 72 doubles per site (SoA double2 chunks)
  void* inv64 = nullptr;    // A^{-1}
  void* blk32 = nullptr;    // A, 72 floats per site (SoA float4 chunks)
  void* inv32 = nullptr;
  void* links32_aos = nullptr;  // [4][V][10] float2, links padded to 80 bytes (ring kernel)
  void* blk32_aos = nullptr;    // [V][72] float, A per site (ring kernel)
  void* inv32_aos = nullptr;    // [V][72] float, A^{-1} per site (ring kernel)
  void* links32_r12 = nullptr;  // [4][6][V] float2, rows 0 and 1 of each link
  void* links_bf16_r12 = nullptr;  // [4][6][V] BF16 pairs, the same rows rounded
  int link_format = 0;          // FP32 operator links: LQCD_LINKS_FP32 (0) or LQCD_LINKS_BF16 (1)
  int* d_err = nullptr;     // device status bitmask
  std::map<std::string, lqcd::Buffer> ws;
  cudaStream_t capture_stream = nullptr;
  lqcd::CycleGraph cycle;
  std::vector<cudaEvent_t> prof_events;  // solver profiling events (4 per Arnoldi step)
  std::map<long long, int> tuned;        // (f64, nrhs, op) -> hopping-kernel variant chosen by lqcd_tune
  void* pinned = nullptr;   // small pinned host staging area
  size_t pinned_bytes = 0;
};

namespace lqcd {

// Error reporting (thread-local message for lqcd_last_error).
lqcd_status set_error(lqcd_status s, const char* fmt, ...);
lqcd_status cuda_error(cudaError_t e, const char* what);
#define LQCD_CUDA(call, what)                              \
  do {                                                     \
    cudaError_t _e = (call);                               \
    if (_e != cudaSuccess) return lqcd::cuda_error(_e, what); \
  } while (0)

// Grow-only named device workspace.
lqcd_status workspace(lqcd_ctx ctx, const char* name, size_t bytes, void** out);
lqcd_status pinned_staging(lqcd_ctx ctx, size_t bytes, void** out);
int* wait_flag(lqcd_ctx ctx);

int site_tile_log2(const lqcd_ctx_s* ctx, int nrhs);
PackedLayout layout_for(const lqcd_ctx_s* ctx, int nrhs);
bool is_device_pointer(const void* p);

// Operator application on packed blocks (used by the apply entry points and the solver).
//   op FULL: in/out full blocks. op SCHUR: in/out odd blocks, tmp = even-half scratch.
lqcd_status apply_operator(lqcd_ctx ctx, int op, bool f64, int nrhs, const void* in, void* out,
                           void* tmp, const int* skip, cudaStream_t stream);
lqcd_status apply_operator_bf16in(lqcd_ctx ctx, int op, int nrhs, const void* in, void* out, void* tmp,
                                  const int* skip, cudaStream_t stream);
// One block GMRES(m) cycle (block_gmres.cu) on D e = r for nrhs <= 16 rhs: x (FP64) += e.
lqcd_status block_gmres_cycle(lqcd_ctx ctx, int op, int nrhs, int m, int64_t n_sys, void* basis, void* tmp_even,
                              const void* r64, void* x64, const double* thr, double* h_res, int* h_flag, int* steps,
                              cudaStream_t st);
lqcd_status schur_prepare(lqcd_ctx ctx, bool f64, int nrhs, const void* b_full, void* bhat_o,
                          void* tmp_even, cudaStream_t stream);
lqcd_status schur_reconstruct(lqcd_ctx ctx, bool f64, int nrhs, const void* b_full, const void* x_o,
                              void* x_full, cudaStream_t stream);

inline long long tune_key(bool f64, int nrhs, int op) { return ((long long)f64 << 40) | ((long long)nrhs << 8) | op; }
inline int tuned_variant(const lqcd_ctx_s* ctx, bool f64, int nrhs, int op) {
  auto it = ctx->tuned.find(tune_key(f64, nrhs, op));
  return it == ctx->tuned.end() ? -1 : it->second;
}

inline size_t packed_elems(const lqcd_ctx_s* ctx, int sites, int nrhs) {
  const size_t ns = sites == LQCD_SITES_FULL ? (size_t)ctx->g.V : (size_t)ctx->g.Vh;
  return ns * 12 * (size_t)nrhs;
}

}  // namespace lqcd
