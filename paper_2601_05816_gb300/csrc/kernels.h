// Internal launcher declarations shared by the library's translation units.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace lqcd {

// pack.cu
// bf16: packed side BF16 pairs, canonical side complex64 (f64 ignored).
cudaError_t launch_spinor_layout(const Geom& g, int sites, int nrhs, int log_s, bool to_packed,
                                 bool f64, const void* in, void* out, cudaStream_t stream, bool bf16 = false);
// Site-major FP32 copies for the ring hopping kernel: links [4][V][10] float2, blocks [V][72] float.
cudaError_t launch_links_aos(int V, const void* links32, void* aos, cudaStream_t s);
cudaError_t launch_blocks_aos(int V, const void* blk32, void* aos, cudaStream_t s);
// Rows 0 and 1 of the FP32 links: [4][6][V] float2 and the same rounded to BF16 pairs.
cudaError_t launch_links_r12(int V, const void* links32, void* r12, void* r12_bf16, cudaStream_t s);
// Column map of the solver's compaction (at most 64 rhs).
struct ColumnMap {
  int col[64];
};
// Gather (dst column k <- src column map.col[k]) or scatter (dst column map.col[k] <- src
// column k) between FP64 packed blocks of n_sites sites with layouts ls and ld.
cudaError_t launch_repack_columns(int64_t n_sites, PackedLayout ls, PackedLayout ld, const ColumnMap& map,
                                  bool scatter, const void* src, void* dst, cudaStream_t stream);
cudaError_t launch_gauge_pack(const Geom& g, int time_bc, const void* U, void* l64, void* l32,
                              cudaStream_t stream);

// clover.cu: site blocks A = (4 + m0) - C and A^{-1}, FP64 then FP32 copies.
// leaf_tmp: device scratch of 6 * 9 * V complex128. err_flag: device int (bitmask).
cudaError_t launch_clover_build(const Geom& g, const void* links64, double m0, double c_sw,
                                void* leaf_tmp, void* blk64, void* inv64, void* blk32, void* inv32,
                                int* err_flag, cudaStream_t stream);
cudaError_t launch_blocks_export(const Geom& g, const void* blk64, void* out, cudaStream_t stream);

// blas.cu: multi-rhs vector kernels on packed blocks of n complex elements
// (rhs of element e is e % nrhs). Reductions go to per-CTA partials, then
// reduce_partials sums them in a fixed order (deterministic).
struct BlasPlan {
  int nrhs;
  int threads;   // multiple of nrhs, <= 256
  int blocks;    // CTAs of the streaming kernels
  int split;     // 1: Gram-Schmidt passes use the warp-split kernel
  int epl;       // 2: the warp-split kernel may put two elements (rhs) per lane (even nrhs <= 64)
  int num_sms;
  // device word that the streaming Gram-Schmidt kernel sets when a pipeline wait gives
  // up (never in correct operation); null: the streaming kernel is not used
  int* wait_flag = nullptr;
};
BlasPlan blas_plan(int64_t n, int nrhs, int num_sms);

// gs_stream_*.cu: the Gram-Schmidt pass with basis tiles staged in shared memory by
// bulk asynchronous copies (FP32 or BF16 basis, nrhs <= 32 or even nrhs <= 64).
// Returns cudaErrorNotSupported (launching nothing) when no layout fits; on success
// the per-CTA partials of *blocks_used CTAs are written.
cudaError_t launch_gs_stream_f32(const BlasPlan& plan, int64_t n, int nvec, const void* basis, int64_t vstride,
                                 void* w, const void* coef, bool update, bool dots, bool norm, void* partials,
                                 const int* skip, cudaStream_t stream, const double* oscale, void* wout,
                                 int* blocks_used);
cudaError_t launch_gs_stream_bf16(const BlasPlan& plan, int64_t n, int nvec, const void* basis,
                                  int64_t vstride, void* w, const void* coef, bool update, bool dots, bool norm,
                                  void* partials, const int* skip, cudaStream_t stream, const double* oscale,
                                  void* wout, int* blocks_used);
// Whether the streaming kernel runs the passes of the delayed re-orthogonalisation (dots +
// norm; update + dots + norm) for basis sizes 1 .. nvec_max (FP32 or BF16 basis).
bool gs_stream_passes_supported_f32(const BlasPlan& plan, int64_t n, int nvec_max);
bool gs_stream_passes_supported_bf16(const BlasPlan& plan, int64_t n, int nvec_max);

// Fused block Gram-Schmidt pass over nvec basis vectors v_i = basis + i * vstride:
//   if update: w <- w - sum_i coef[i][r] v_i   (coef: device double2 [nvec][nrhs])
//   if dots:   out[i][r] = <v_i, w>  (after the update)
//   if norm:   out[nvec][r] = ||w||^2 (real part)
// out: device double2 [nvec + 1][nrhs]; partials: device scratch double2
// [plan.blocks][nvec + 1][nrhs]. skip: optional device flag (return when set).
//   oscale: optional device double [nrhs]; the updated w is multiplied by it before the store
//   (dots and norm refer to the unscaled w). With neither dots nor norm no reduction runs.
//   basis_bf16: basis stored as BF16 pairs (FP32 arithmetic, w in FP32; needs plan.split);
//   wout: optional, the scaled updated w is stored there (in the basis storage type) instead of in w.
cudaError_t launch_gs_pass(bool f64, const BlasPlan& plan, int64_t n, int nvec, const void* basis,
                           int64_t vstride, void* w, const void* coef, bool update, bool dots,
                           bool norm, void* partials, void* out, const int* skip,
                           cudaStream_t stream, const double* oscale = nullptr, bool basis_bf16 = false,
                           void* wout = nullptr);

// r = b - t (b, r FP64; t FP64, or FP32 when t_f32) with out[0][r] = ||r||^2.
cudaError_t launch_sub_norm(const BlasPlan& plan, int64_t n, const void* b, const void* t, void* r,
                            void* partials, void* out, cudaStream_t stream, bool t_f32 = false);
// out = (FP32) (a - b), a and b FP64.
cudaError_t launch_diff_to_f32(int64_t n, const void* a, const void* b, void* out, cudaStream_t stream);
// ||v||^2 per rhs, out[0][r]; v in FP64 or FP32.
cudaError_t launch_norm2(bool f64, const BlasPlan& plan, int64_t n, const void* v, void* partials,
                         void* out, cudaStream_t stream);
// dst[e] = (dst precision) (src[e] * scale[r]); src FP64, dst FP64, FP32 or BF16 pairs.
cudaError_t launch_scale_convert(bool dst_f64, int64_t n, int nrhs, const void* src,
                                 const double* scale, void* dst, cudaStream_t stream, bool dst_bf16 = false);
// v[e] *= scale[r] in place (v FP64 or FP32).
cudaError_t launch_scale_inplace(bool f64, int64_t n, int nrhs, void* v, const double* scale,
                                 const int* skip, cudaStream_t stream);
// x[e] += sum_{i < *kmax} y[i][r] v_i[e]; x FP64, basis FP64 or FP32 (sum in basis precision).
cudaError_t launch_update_x(bool basis_f64, int64_t n, int nrhs, int nvec_max, const void* basis,
                            int64_t vstride, const void* y, const int* kmax, void* x,
                            cudaStream_t stream, bool basis_bf16 = false);
// force.cu: gamma5 = diag(-1, -1, 1, 1) in place on an FP64 packed block of n complex
// elements (nrhs rhs, site tile 2^log_s).
cudaError_t launch_gamma5_packed(int64_t n, int nrhs, int log_s, void* v, cudaStream_t s);
// Widen / narrow copies between FP64 and FP32 packed blocks.
cudaError_t launch_convert(bool to_f64, int64_t n, const void* src, void* dst, cudaStream_t stream);

// gmres.cu: per-rhs small dense work of Algorithm 2 in FP64 on the device.
struct GmresState {
  int m, nrhs;
  double2* H;        // [nrhs][m][m + 1]: column j of the rotated Hessenberg matrix
  double* cs;        // [nrhs][m]
  double2* sn;       // [nrhs][m]
  double2* gamma;    // [nrhs][m + 1]
  double2* y;        // [m][nrhs]
  double* thr;       // [nrhs] absolute stop threshold of the cycle
  double* scale;     // [nrhs] 1 / beta for the next basis vector (0 = inactive)
  int* active;       // [nrhs]
  int* done;         // [nrhs] cycle finished for this rhs
  int* k;            // [nrhs] Arnoldi steps taken in this cycle
  int* all_done;     // [1]
  int* kmax;         // [1]
};
// init: gamma = (beta0, 0, ...), done = !active, scale = active / beta0.
cudaError_t launch_cycle_init(const GmresState& s, const double* beta0, cudaStream_t stream);
// step j: column from h1 (+ h2 when h2 != null) and ||w||^2 = hn[j + 1][r], rotations, gamma, stop test.
// With pythag, ||w||^2 = hn[j + 1][r] - sum_i |h2[i][r]|^2 (hn holds ||w'||^2 before the second
// Gram-Schmidt correction h2, which is orthogonal to the final w).
cudaError_t launch_givens(const GmresState& s, int j, const void* h1, const void* h2, const void* hn,
                          bool pythag, cudaStream_t stream);
cudaError_t launch_backsub(const GmresState& s, cudaStream_t stream);

// dslash_f32.cu / dslash_f64.cu: see dslash.cuh.

}  // namespace lqcd
