// Variant tables and dispatch of the multi-rhs hopping kernel.
#include "dslash_async.cuh"
#include "dslash_ring.cuh"
#include "dslash_pipe.cuh"

namespace lqcd {

namespace {
// {rhs per thread, threads per CTA, min CTAs per SM, cp.async stages (0 = direct loads),
//  batched loads, persistent chunk loop, rhs count fixed at compile time, L1 prefetch distance,
//  ring kernel warps per CTA, ring slots per warp, two-row links, blocked rows + x, y, z, t order,
//  pipelined kernel stages}
const DslashVariant kF32[] = {{2, 128, 1, 0, 0, 0}, {2, 128, 4, 0, 0, 0}, {1, 128, 1, 0, 0, 0}, {1, 128, 6, 0, 0, 0}, {1, 256, 1, 0, 0, 0}, {2, 256, 2, 0, 0, 0}, {2, 128, 1, 2, 0, 0}, {2, 128, 4, 0, 1, 0}, {2, 64, 8, 0, 1, 0}, {2, 128, 4, 0, 0, 1}, {2, 128, 4, 0, 1, 1}, {2, 256, 2, 0, 0, 1}, {1, 128, 6, 0, 0, 1},
                             {2, 128, 4, 0, 0, 0, 16}, {2, 256, 2, 0, 0, 0, 16},
                             {2, 128, 4, 0, 0, 0, 16, 1}, {2, 128, 4, 0, 0, 0, 16, 2}, {2, 256, 2, 0, 0, 0, 16, 1},
                             {2, 128, 4, 0, 0, 0, 32}, {2, 128, 4, 0, 0, 0, 32, 1},
                             {2, 128, 4, 0, 0, 0, 64}, {2, 128, 4, 0, 0, 0, 64, 1},
                             // bulk-copy ring kernel (dslash_ring.cuh): CTAs per SM (minb), warps per CTA,
                             // ring slots per warp
                             {2, 256, 1, 0, 0, 0, 16, 0, 8, 3}, {2, 384, 1, 0, 0, 0, 16, 0, 12, 2},
                             {2, 448, 1, 0, 0, 0, 16, 0, 14, 2}, {2, 224, 2, 0, 0, 0, 16, 0, 7, 2},
                             {2, 192, 2, 0, 0, 0, 16, 0, 6, 2}, {2, 512, 1, 0, 0, 0, 16, 0, 16, 1},
                             {2, 384, 1, 0, 0, 0, 32, 0, 12, 2}, {2, 224, 2, 0, 0, 0, 32, 0, 7, 2},
                             {2, 384, 1, 0, 0, 0, 64, 0, 12, 2}, {2, 224, 2, 0, 0, 0, 64, 0, 7, 2},
                             {2, 256, 1, 0, 0, 0, 64, 0, 8, 3},
                             // two-row FP32 links (third row rebuilt)
                             {1, 256, 1, 0, 0, 0, 0, 0, 0, 0, 1}, {2, 256, 2, 0, 0, 0, 0, 0, 0, 0, 1},
                             {2, 128, 4, 0, 0, 0, 0, 0, 0, 0, 1}, {2, 256, 2, 0, 0, 1, 0, 0, 0, 0, 1},
                             {2, 128, 4, 0, 0, 0, 16, 2, 0, 0, 1},
                             // blocked rows per CTA, directions x, y, z, t
                             {2, 512, 1, 0, 0, 0, 16, 0, 0, 0, 0, 1}, {2, 512, 1, 0, 0, 0, 16, 2, 0, 0, 0, 1},
                             {2, 256, 2, 0, 0, 0, 16, 2, 0, 0, 0, 1}, {2, 512, 1, 0, 0, 0, 32, 2, 0, 0, 0, 1},
                             // pipelined kernel (dslash_pipe.cuh): operands one or two directions ahead in
                             // shared memory, copied by each thread with cp.async
                             {2, 128, 4, 0, 0, 0, 16, 0, 0, 0, 0, 0, 2}, {2, 128, 2, 0, 0, 0, 16, 0, 0, 0, 0, 0, 3},
                             {2, 256, 2, 0, 0, 0, 16, 0, 0, 0, 0, 0, 2}, {2, 128, 4, 0, 0, 0, 32, 0, 0, 0, 0, 0, 2},
                             {2, 128, 4, 0, 0, 0, 64, 0, 0, 0, 0, 0, 2}};
const DslashVariant kF64[] = {{1, 128, 1, 0, 0, 0}, {1, 128, 4, 0, 0, 0}, {1, 256, 1, 0, 0, 0}, {1, 64, 1, 0, 0, 0}, {1, 128, 1, 2, 0, 0}, {1, 128, 4, 0, 1, 0}, {1, 128, 4, 0, 0, 1}};
}  // namespace

extern template cudaError_t launch_dslash_variant<float, 2, 128, 1, false, false>(const DslashArgs<float>&, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_variant<float, 2, 128, 4, false, false>(const DslashArgs<float>&, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_variant<float, 1, 128, 1, false, false>(const DslashArgs<float>&, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_variant<float, 1, 128, 6, false, false>(const DslashArgs<float>&, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_variant<float, 1, 256, 1, false, false>(const DslashArgs<float>&, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_variant<float, 2, 256, 2, false, false>(const DslashArgs<float>&, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_async_variant<float, 2, 128, 1, 2>(const DslashArgs<float>&, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_variant<float, 2, 128, 4, true, false>(const DslashArgs<float>&, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_variant<float, 2, 64, 8, true, false>(const DslashArgs<float>&, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_variant<float, 2, 128, 4, false, true>(const DslashArgs<float>&, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_variant<float, 2, 128, 4, true, true>(const DslashArgs<float>&, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_variant<float, 2, 256, 2, false, true>(const DslashArgs<float>&, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_variant<float, 1, 128, 6, false, true>(const DslashArgs<float>&, int, int, cudaStream_t);
#define LQCD_EXTERN_NRHS(MAXT, MINB, NRHS, PF)                                                             \
  extern template cudaError_t launch_dslash_variant<float, 2, MAXT, MINB, false, false, float2, float2, NRHS, PF>( \
      const DslashArgs<float>&, int, int, cudaStream_t);
LQCD_EXTERN_NRHS(128, 4, 16, 0)
LQCD_EXTERN_NRHS(256, 2, 16, 0)
LQCD_EXTERN_NRHS(128, 4, 16, 1)
LQCD_EXTERN_NRHS(128, 4, 16, 2)
LQCD_EXTERN_NRHS(256, 2, 16, 1)
LQCD_EXTERN_NRHS(128, 4, 32, 0)
LQCD_EXTERN_NRHS(128, 4, 32, 1)
LQCD_EXTERN_NRHS(128, 4, 64, 0)
LQCD_EXTERN_NRHS(128, 4, 64, 1)
#undef LQCD_EXTERN_NRHS
#define LQCD_EXTERN_LF(NR, MAXT, MINB, LOOP, NRHS, PF, LF)                                                  \
  extern template cudaError_t launch_dslash_variant<float, NR, MAXT, MINB, false, LOOP, float2, float2, NRHS, PF, LF>( \
      const DslashArgs<float>&, int, int, cudaStream_t);
LQCD_EXTERN_LF(1, 256, 1, false, 0, 0, 1)
LQCD_EXTERN_LF(2, 256, 2, false, 0, 0, 1)
LQCD_EXTERN_LF(2, 128, 4, false, 0, 0, 1)
LQCD_EXTERN_LF(2, 256, 2, true, 0, 0, 1)
LQCD_EXTERN_LF(2, 128, 4, false, 16, 2, 1)
LQCD_EXTERN_LF(1, 256, 1, false, 0, 0, 2)
LQCD_EXTERN_LF(2, 128, 4, false, 0, 0, 2)
LQCD_EXTERN_LF(2, 256, 2, true, 0, 0, 2)
LQCD_EXTERN_LF(2, 128, 4, false, 16, 2, 2)
#undef LQCD_EXTERN_LF
#define LQCD_EXTERN_ORD(NR, MAXT, MINB, NRHS, PF)                                                              \
  extern template cudaError_t launch_dslash_variant<float, NR, MAXT, MINB, false, false, float2, float2, NRHS, PF, 0, 1>( \
      const DslashArgs<float>&, int, int, cudaStream_t);
LQCD_EXTERN_ORD(2, 512, 1, 16, 0)
LQCD_EXTERN_ORD(2, 512, 1, 16, 2)
LQCD_EXTERN_ORD(2, 256, 2, 16, 2)
LQCD_EXTERN_ORD(2, 512, 1, 32, 2)
#undef LQCD_EXTERN_ORD
extern template cudaError_t launch_dslash_pipe<16, 128, 4, 2>(const DslashArgs<float>&, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_pipe<16, 128, 2, 3>(const DslashArgs<float>&, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_pipe<16, 256, 2, 2>(const DslashArgs<float>&, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_pipe<32, 128, 4, 2>(const DslashArgs<float>&, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_pipe<64, 128, 4, 2>(const DslashArgs<float>&, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_ring<16>(const DslashArgs<float>&, int, int, int, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_ring<32>(const DslashArgs<float>&, int, int, int, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_ring<64>(const DslashArgs<float>&, int, int, int, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_variant<double, 1, 128, 1, false, false>(const DslashArgs<double>&, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_variant<double, 1, 128, 4, false, false>(const DslashArgs<double>&, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_variant<double, 1, 256, 1, false, false>(const DslashArgs<double>&, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_variant<double, 1, 64, 1, false, false>(const DslashArgs<double>&, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_async_variant<double, 1, 128, 1, 2>(const DslashArgs<double>&, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_variant<double, 1, 128, 4, true, false>(const DslashArgs<double>&, int, int, cudaStream_t);
extern template cudaError_t launch_dslash_variant<double, 1, 128, 4, false, true>(const DslashArgs<double>&, int, int, cudaStream_t);

int dslash_variant_count(bool f64) { return f64 ? (int)(sizeof(kF64) / sizeof(kF64[0])) : (int)(sizeof(kF32) / sizeof(kF32[0])); }

DslashVariant dslash_variant(bool f64, int idx) { return f64 ? kF64[idx] : kF32[idx]; }

bool dslash_variant_ok(bool f64, int idx, int nrhs) {
  if (idx < 0 || idx >= dslash_variant_count(f64)) return false;
  const DslashVariant v = dslash_variant(f64, idx);
  if (v.nrhs_fixed > 0 && nrhs != v.nrhs_fixed) return false;
  return nrhs % v.nr == 0 && nrhs / v.nr <= v.threads;
}

int dslash_default_variant(bool f64, int nrhs) {
  if (f64) return nrhs <= 128 ? 0 : 2;
  if (nrhs % 2 == 0 && nrhs / 2 <= 128) return 1;
  return nrhs <= 128 ? 2 : 4;
}

template <>
cudaError_t launch_dslash<float>(const DslashArgs<float>& a, int self_mode, int post_mode, int variant,
                                 cudaStream_t s) {
  if (a.link_format == 2) {
    // BF16 two-row links (a storage choice of the context, not a tuned variant): a fixed
    // launch shape per rhs count
    const int n = a.lay.nrhs;
    if (n == 16 && a.lay.log_s == 0)
      return launch_dslash_variant<float, 2, 128, 4, false, false, float2, float2, 16, 2, 2>(a, self_mode, post_mode, s);
    if (n % 2 == 0 && n / 2 <= 128) {
      if (n <= 4) return launch_dslash_variant<float, 2, 256, 2, false, true, float2, float2, 0, 0, 2>(a, self_mode, post_mode, s);
      return launch_dslash_variant<float, 2, 128, 4, false, false, float2, float2, 0, 0, 2>(a, self_mode, post_mode, s);
    }
    return launch_dslash_variant<float, 1, 256, 1, false, false, float2, float2, 0, 0, 2>(a, self_mode, post_mode, s);
  }
  if (!dslash_variant_ok(false, variant, a.lay.nrhs)) variant = dslash_default_variant(false, a.lay.nrhs);
  const DslashVariant v = kF32[variant];
  if (v.ring_warps > 0) {
    const int cps = v.minb;  // resident CTAs per SM the variant is built for
    if (v.nrhs_fixed == 16) return launch_dslash_ring<16>(a, self_mode, post_mode, v.ring_warps, v.ring_slots, cps, s);
    if (v.nrhs_fixed == 32) return launch_dslash_ring<32>(a, self_mode, post_mode, v.ring_warps, v.ring_slots, cps, s);
    if (v.nrhs_fixed == 64) return launch_dslash_ring<64>(a, self_mode, post_mode, v.ring_warps, v.ring_slots, cps, s);
    return cudaErrorInvalidValue;
  }
  switch (variant) {
    case 0: return launch_dslash_variant<float, 2, 128, 1, false, false>(a, self_mode, post_mode, s);
    case 1: return launch_dslash_variant<float, 2, 128, 4, false, false>(a, self_mode, post_mode, s);
    case 2: return launch_dslash_variant<float, 1, 128, 1, false, false>(a, self_mode, post_mode, s);
    case 3: return launch_dslash_variant<float, 1, 128, 6, false, false>(a, self_mode, post_mode, s);
    case 4: return launch_dslash_variant<float, 1, 256, 1, false, false>(a, self_mode, post_mode, s);
    case 5: return launch_dslash_variant<float, 2, 256, 2, false, false>(a, self_mode, post_mode, s);
    case 6: return launch_dslash_async_variant<float, 2, 128, 1, 2>(a, self_mode, post_mode, s);
    case 7: return launch_dslash_variant<float, 2, 128, 4, true, false>(a, self_mode, post_mode, s);
    case 8: return launch_dslash_variant<float, 2, 64, 8, true, false>(a, self_mode, post_mode, s);
    case 9: return launch_dslash_variant<float, 2, 128, 4, false, true>(a, self_mode, post_mode, s);
    case 10: return launch_dslash_variant<float, 2, 128, 4, true, true>(a, self_mode, post_mode, s);
    case 11: return launch_dslash_variant<float, 2, 256, 2, false, true>(a, self_mode, post_mode, s);
    case 12: return launch_dslash_variant<float, 1, 128, 6, false, true>(a, self_mode, post_mode, s);
#define LQCD_CASE_NRHS(IDX, MAXT, MINB, NRHS, PF) \
  case IDX: return launch_dslash_variant<float, 2, MAXT, MINB, false, false, float2, float2, NRHS, PF>(a, self_mode, post_mode, s);
    LQCD_CASE_NRHS(13, 128, 4, 16, 0)
    LQCD_CASE_NRHS(14, 256, 2, 16, 0)
    LQCD_CASE_NRHS(15, 128, 4, 16, 1)
    LQCD_CASE_NRHS(16, 128, 4, 16, 2)
    LQCD_CASE_NRHS(17, 256, 2, 16, 1)
    LQCD_CASE_NRHS(18, 128, 4, 32, 0)
    LQCD_CASE_NRHS(19, 128, 4, 32, 1)
    LQCD_CASE_NRHS(20, 128, 4, 64, 0)
    LQCD_CASE_NRHS(21, 128, 4, 64, 1)
#undef LQCD_CASE_NRHS
    case 33: return launch_dslash_variant<float, 1, 256, 1, false, false, float2, float2, 0, 0, 1>(a, self_mode, post_mode, s);
    case 34: return launch_dslash_variant<float, 2, 256, 2, false, false, float2, float2, 0, 0, 1>(a, self_mode, post_mode, s);
    case 35: return launch_dslash_variant<float, 2, 128, 4, false, false, float2, float2, 0, 0, 1>(a, self_mode, post_mode, s);
    case 36: return launch_dslash_variant<float, 2, 256, 2, false, true, float2, float2, 0, 0, 1>(a, self_mode, post_mode, s);
    case 37: return launch_dslash_variant<float, 2, 128, 4, false, false, float2, float2, 16, 2, 1>(a, self_mode, post_mode, s);
    case 38: return launch_dslash_variant<float, 2, 512, 1, false, false, float2, float2, 16, 0, 0, 1>(a, self_mode, post_mode, s);
    case 39: return launch_dslash_variant<float, 2, 512, 1, false, false, float2, float2, 16, 2, 0, 1>(a, self_mode, post_mode, s);
    case 40: return launch_dslash_variant<float, 2, 256, 2, false, false, float2, float2, 16, 2, 0, 1>(a, self_mode, post_mode, s);
    case 41: return launch_dslash_variant<float, 2, 512, 1, false, false, float2, float2, 32, 2, 0, 1>(a, self_mode, post_mode, s);
    case 42: return launch_dslash_pipe<16, 128, 4, 2>(a, self_mode, post_mode, s);
    case 43: return launch_dslash_pipe<16, 128, 2, 3>(a, self_mode, post_mode, s);
    case 44: return launch_dslash_pipe<16, 256, 2, 2>(a, self_mode, post_mode, s);
    case 45: return launch_dslash_pipe<32, 128, 4, 2>(a, self_mode, post_mode, s);
    case 46: return launch_dslash_pipe<64, 128, 4, 2>(a, self_mode, post_mode, s);
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_dslash<double>(const DslashArgs<double>& a, int self_mode, int post_mode, int variant,
                                 cudaStream_t s) {
  if (!dslash_variant_ok(true, variant, a.lay.nrhs)) variant = dslash_default_variant(true, a.lay.nrhs);
  switch (variant) {
    case 0: return launch_dslash_variant<double, 1, 128, 1, false, false>(a, self_mode, post_mode, s);
    case 1: return launch_dslash_variant<double, 1, 128, 4, false, false>(a, self_mode, post_mode, s);
    case 2: return launch_dslash_variant<double, 1, 256, 1, false, false>(a, self_mode, post_mode, s);
    case 3: return launch_dslash_variant<double, 1, 64, 1, false, false>(a, self_mode, post_mode, s);
    case 4: return launch_dslash_async_variant<double, 1, 128, 1, 2>(a, self_mode, post_mode, s);
    case 5: return launch_dslash_variant<double, 1, 128, 4, true, false>(a, self_mode, post_mode, s);
    case 6: return launch_dslash_variant<double, 1, 128, 4, false, true>(a, self_mode, post_mode, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lqcd
