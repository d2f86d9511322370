// Allocation-free variant of the odd-even Schur operator apply.
//
// lqcd_apply_packed(LQCD_OP_SCHUR) keeps its intermediate block
// t_e = A_ee^{-1} D_eo psi_o in library workspace that it allocates with
// cudaMalloc on first use. Some callers cannot let a library allocate device
// memory at that point: applications whose own pool allocator has already
// reserved nearly all of the GPU's memory (a cudaMalloc from the library would
// then fail), applications that need a fixed device-memory footprint known
// before they start, and latency-critical loops that cannot accept the device
// synchronisation a cudaMalloc/cudaFree may cause. For them this file provides
// lqcd_apply_schur_noalloc, which keeps t_e in a statically sized device array
// that exists from module load until process exit, and calls no allocating
// routine (no cudaMalloc, cudaFree, or library call that allocates).
#include <mutex>

#include "ctx.h"

namespace {

// Scratch of the allocation-free Schur apply. Every GPU that loads the library
// holds this array until the process exits.
constexpr size_t kNoallocScratchBytes = (size_t)64 << 20;  // 64 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void* g_scratch_address[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on the current device, looked up once per
// device with that device current. In host code the symbol itself is only a
// host-side stand-in and must never be passed to a kernel. The current device
// must be the one holding the context's fields (the device that was current at
// lqcd_set_gauge): the kernels read the links there and write the scratch array
// of the current device.
lqcd_status scratch_address(int ctx_device, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return lqcd::cuda_error(e, "lqcd_apply_schur_noalloc: cudaGetDevice");
  if (dev != ctx_device)
    return lqcd::set_error(LQCD_ERR_STATE,
                           "lqcd_apply_schur_noalloc: device %d is current but the context's fields live on "
                           "device %d; make that device current first", dev, ctx_device);
  if (dev < 0 || dev >= kMaxDevices)
    return lqcd::set_error(LQCD_ERR_ARG, "lqcd_apply_schur_noalloc: device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (g_scratch_address[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return lqcd::cuda_error(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                              "lqcd_apply_schur_noalloc: cudaGetSymbolAddress(scratch)");
    g_scratch_address[dev] = p;
  }
  *out = g_scratch_address[dev];
  return LQCD_OK;
}

}  // namespace

extern "C" {

size_t lqcd_noalloc_scratch_bytes(void) { return kNoallocScratchBytes; }

lqcd_status lqcd_apply_schur_noalloc(lqcd_ctx ctx, lqcd_dtype dtype, int nrhs, const void* in, void* out,
                                     void* stream) {
  if (ctx == nullptr) return lqcd::set_error(LQCD_ERR_ARG, "lqcd_apply_schur_noalloc: null context");
  if (!ctx->have_gauge || !ctx->have_blocks)
    return lqcd::set_error(LQCD_ERR_STATE,
                           "lqcd_apply_schur_noalloc: lqcd_set_gauge and lqcd_set_clover must be called first");
  if ((dtype != LQCD_C64 && dtype != LQCD_C128) || nrhs < 1 || nrhs > 256 || in == nullptr || out == nullptr ||
      in == out)
    return lqcd::set_error(LQCD_ERR_ARG, "lqcd_apply_schur_noalloc: bad arguments");
  const size_t need = (size_t)ctx->g.Vh * 12 * (size_t)nrhs * (dtype == LQCD_C128 ? 16 : 8);
  if (need > kNoallocScratchBytes)
    return lqcd::set_error(LQCD_ERR_ARG,
                           "lqcd_apply_schur_noalloc: the intermediate block needs %zu bytes (V/2 * 12 * nrhs "
                           "complex), more than the fixed %zu-byte scratch; use lqcd_apply_packed instead",
                           need, kNoallocScratchBytes);
  void* scratch = nullptr;
  lqcd_status st = scratch_address(ctx->device, &scratch);
  if (st != LQCD_OK) return st;
  // Pass A overwrites every element of the scratch block before pass B reads it,
  // so nothing left over from an earlier call is ever used.
  return lqcd::apply_operator(ctx, LQCD_OP_SCHUR, dtype == LQCD_C128, nrhs, in, out, scratch, nullptr,
                              (cudaStream_t)stream);
}

}  // extern "C"
