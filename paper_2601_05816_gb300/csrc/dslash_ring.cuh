// Multi-rhs hopping kernel with a per-warp shared-memory ring fed by bulk copies
// (Sec. III-A-1, Algorithm 1 with the rhs loop inside the site loop, Eq. (2)).
//
// Same operator as dslash_kernel (dslash.cuh): out(x) = POST(SELF(x) + c_hop H(x))
// for FP32 blocks whose rhs count NRHS is 16, 32 or 64 (site tile of one site, so a
// site's 12 * NRHS complex numbers are one contiguous run). What changes is where
// the operands wait while they are in flight. In dslash_kernel every byte of a
// neighbour spinor lands in a register, so the bytes in flight per SM are bounded
// by the register file, and the kernel is latency-bound. Here each warp owns a ring
// of K slots in shared memory; one slot holds, for the warp's TPW = 64 / NRHS target
// sites, one hopping direction's operands: the TPW neighbour spinors (all rhs) and
// the TPW links (80-byte padded copies). A ninth slot per target group holds the
// site-local operands (the self-term spinor and the clover block A or A^-1). Lane 0
// posts the slot's byte count on its mbarrier and lanes 0..TPW-1 issue one bulk copy
// per spinor and per link; the warp then computes the slot issued K-1 steps earlier.
// A slot is refilled as soon as the warp has read it (the warp is its own producer,
// so program order and __syncwarp replace an "empty" barrier), so K-1 slots of every
// warp are in flight while it computes: up to W (K-1) 6.4 KB per SM, independent of
// registers. Each lane then does the same arithmetic as dslash_kernel for its two rhs
// of one target site, reading the operands from shared memory.
//
// Every wait is bounded (bulk::mbar_wait_bounded); one that gives up sets *err, the
// warp waits (bounded) for its copies in flight and returns.
#pragma once
#include "bulk_async.cuh"
#include "dslash.cuh"

namespace lqcd {
namespace ring {

using namespace bulk;

constexpr int kLinkStride = 10;          // complex entries per padded link: 9 + 1 unused
constexpr uint32_t kLinkBytes = 80;      // 16-byte multiple, as bulk copies need
constexpr uint32_t kBlockBytes = 72 * 4; // one site's A or A^-1 in FP32

template <int NRHS>
struct Shape {
  static_assert(NRHS == 16 || NRHS == 32 || NRHS == 64, "ring kernel: 16, 32 or 64 rhs");
  static constexpr int G = NRHS / 2;               // lanes of one target site (two rhs per lane)
  static constexpr int TPW = 32 / G;               // target sites per warp
  static constexpr uint32_t SP = 12u * NRHS * 8u;  // bytes of one site's spinor, all rhs
  static constexpr uint32_t EXTRA = TPW * kBlockBytes;  // links or site blocks of the slot
  static constexpr uint32_t SLOT = (TPW * SP + EXTRA + 127u) / 128u * 128u;
};

template <int NRHS>
__host__ __device__ constexpr size_t smem_bytes(int warps, int slots) {
  return (size_t)warps * slots * Shape<NRHS>::SLOT + (size_t)warps * slots * sizeof(uint64_t);
}

// Site number of the neighbour in hopping direction k = 0..7 (mu = k / 2, forward for even k).
__device__ __forceinline__ int neighbour_lex_k(const Geom& g, const Coord& c, int k) {
  switch (k) {
    case 0: return neighbour_lex<0, +1>(g, c);
    case 1: return neighbour_lex<0, -1>(g, c);
    case 2: return neighbour_lex<1, +1>(g, c);
    case 3: return neighbour_lex<1, -1>(g, c);
    case 4: return neighbour_lex<2, +1>(g, c);
    case 5: return neighbour_lex<2, -1>(g, c);
    case 6: return neighbour_lex<3, +1>(g, c);
    default: return neighbour_lex<3, -1>(g, c);
  }
}

// Target site of producer lane l (< TPW) of a target group: parity, checkerboard index,
// coordinates. Computed once per group (the divisions of site_coords), reused for its slots.
struct ProdSite {
  int group;  // first target index of the group these values belong to (-1: none yet)
  int p, cb;
  Coord c;
};

// The operands of slot s (0..7: hopping direction s; 8: site-local operands) of the target
// group starting at `first`, posted on the slot's barrier. Called by the whole warp.
template <int SELF, int POST, int NRHS>
__device__ __forceinline__ void produce(const DslashArgs<float>& a, unsigned char* slot, uint64_t* bar, int first,
                                        int s, int lane, ProdSite& ps) {
  using Sh = Shape<NRHS>;
  constexpr bool SELF_IN = SELF != SELF_NONE;
  constexpr bool BLOCK = SELF == SELF_BLOCK || POST == POST_BLOCKINV;
  const int nvalid = min(Sh::TPW, a.n_target - first);
  const uint32_t bytes = s < 8 ? (uint32_t)nvalid * (Sh::SP + kLinkBytes)
                               : (uint32_t)nvalid * ((SELF_IN ? Sh::SP : 0u) + (BLOCK ? kBlockBytes : 0u));
  if (lane == 0) mbar_expect_tx(bar, bytes);
  __syncwarp();
  if (lane < nvalid) {
    if (ps.group != first) {
      const int site = first + lane;
      if (a.full) {
        ps.p = site >= a.g.Vh ? 1 : 0;
        ps.cb = site - ps.p * a.g.Vh;
      } else {
        ps.p = a.target_parity;
        ps.cb = site;
      }
      ps.c = site_coords(a.g, ps.p, ps.cb);
      ps.group = first;
    }
    const int p = ps.p, cb = ps.cb;
    if (s < 8) {
      const int ncb = neighbour_lex_k(a.g, ps.c, s) >> 1;
      const float2* hin = a.hop_in + (a.full ? (int64_t)(1 - p) * a.half_elems : 0);
      bulk_load(slot + (size_t)lane * Sh::SP, hin + (int64_t)ncb * 12 * NRHS, Sh::SP, bar);
      const int mu = s >> 1;
      const int link_site = (s & 1) == 0 ? p * a.g.Vh + cb : (1 - p) * a.g.Vh + ncb;
      const float2* lk = static_cast<const float2*>(a.links_aos) + ((int64_t)mu * a.g.V + link_site) * kLinkStride;
      bulk_load(slot + (size_t)Sh::TPW * Sh::SP + (size_t)lane * kLinkBytes, lk, kLinkBytes, bar);
    } else {
      const int64_t base = a.full ? (int64_t)p * a.half_elems : 0;
      if (SELF_IN)
        bulk_load(slot + (size_t)lane * Sh::SP, a.self_in + base + (int64_t)cb * 12 * NRHS, Sh::SP, bar);
      if (BLOCK) {
        const float* blk = static_cast<const float*>(SELF == SELF_BLOCK ? a.blocks_aos : a.blocks_inv_aos);
        bulk_load(slot + (size_t)Sh::TPW * Sh::SP + (size_t)lane * kBlockBytes,
                  blk + (int64_t)(p * a.g.Vh + cb) * 72, kBlockBytes, bar);
      }
    }
  }
}

// Spinor components of one slot for this lane (target t, rhs r0, r0 + 1): shared-memory loads.
template <int NRHS>
__device__ __forceinline__ void lds_spinor(const unsigned char* slot, int t, int r0, int c0, MC<float, 2>* v) {
  const float2* sp = reinterpret_cast<const float2*>(slot + (size_t)t * Shape<NRHS>::SP);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float4 q = *reinterpret_cast<const float4*>(sp + (c0 + k) * NRHS + r0);
    v[k].re[0] = q.x; v[k].im[0] = q.y; v[k].re[1] = q.z; v[k].im[1] = q.w;
  }
}

template <int NRHS, int MU, int DIR>
__device__ __forceinline__ void consume_dir(const unsigned char* slot, int t, int r0, MC<float, 2> acc[12]) {
  using Sh = Shape<NRHS>;
  const float4* lk = reinterpret_cast<const float4*>(slot + (size_t)Sh::TPW * Sh::SP + (size_t)t * kLinkBytes);
  float2 u[9];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float4 q = lk[k];
    u[2 * k] = make_float2(q.x, q.y);
    u[2 * k + 1] = make_float2(q.z, q.w);
  }
  u[8] = reinterpret_cast<const float2*>(lk)[8];
  MC<float, 2> up[6], dn[6];
  lds_spinor<NRHS>(slot, t, r0, 0, up);
  lds_spinor<NRHS>(slot, t, r0, 6, dn);
  hop_compute<float, 2, MU, DIR>(u, up, dn, acc);
}

// Wait for slot seq (all lanes observe the barrier; the warp agrees on the outcome).
__device__ __forceinline__ bool wait_slot(uint64_t* bars, int K, int seq) {
  const bool mine = mbar_wait_bounded(&bars[seq % K], (uint32_t)(seq / K) & 1u);
  return __all_sync(0xffffffffu, mine);
}

template <int SELF, int POST, int NRHS, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) dslash_ring_kernel(const DslashArgs<float> a) {
  using Sh = Shape<NRHS>;
  constexpr bool HAS_SITE = SELF != SELF_NONE || POST == POST_BLOCKINV;
  constexpr int NSLOT = 8 + (HAS_SITE ? 1 : 0);
  if (a.skip != nullptr && *a.skip != 0) return;
  extern __shared__ __align__(128) unsigned char smem[];
  const int K = a.ring_slots;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int W = blockDim.x >> 5;
  unsigned char* ring = smem + (size_t)warp * K * Sh::SLOT;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)W * K * Sh::SLOT) + warp * K;
  if (lane == 0) {
    for (int k = 0; k < K; ++k) mbar_init(&bars[k], 1);
    fence_proxy_async();  // the initialised barriers are seen by the copy engine
  }
  __syncwarp();

  const int n_tasks = (a.n_target + Sh::TPW - 1) / Sh::TPW;
  const int task0 = blockIdx.x * W + warp;
  const int tstride = gridDim.x * W;
  const int my_tasks = task0 < n_tasks ? (n_tasks - 1 - task0) / tstride + 1 : 0;
  const int total = my_tasks * NSLOT;
  const int t = lane / Sh::G;         // this lane's target in the group
  const int r0 = (lane % Sh::G) * 2;  // and its two rhs

  int issued = 0;
  ProdSite ps;
  ps.group = -1;
  auto post = [&](int seq) {
    const int it = seq / NSLOT;
    produce<SELF, POST, NRHS>(a, ring + (size_t)(seq % K) * Sh::SLOT, &bars[seq % K],
                              (task0 + it * tstride) * Sh::TPW, seq - it * NSLOT, lane, ps);
  };
  for (; issued < K - 1 && issued < total; ++issued) post(issued);

  bool ok = true;
  int seq = 0;
  // next slot: refill the buffer read in the previous step, then wait for this one
  auto advance = [&]() -> const unsigned char* {
    if (issued < total) {
      __syncwarp();
      fence_proxy_async();
      post(issued);
    }
    ++issued;
    if (!wait_slot(bars, K, seq)) {
      ok = false;
      return nullptr;
    }
    return ring + (size_t)(seq++ % K) * Sh::SLOT;
  };

  for (int it = 0; it < my_tasks && ok; ++it) {
    const int site = (task0 + it * tstride) * Sh::TPW + t;
    MC<float, 2> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) mc_zero(acc[k]);
    const unsigned char* sl;
    if ((sl = advance()) == nullptr) break;
    consume_dir<NRHS, 0, +1>(sl, t, r0, acc);
    if ((sl = advance()) == nullptr) break;
    consume_dir<NRHS, 0, -1>(sl, t, r0, acc);
    if ((sl = advance()) == nullptr) break;
    consume_dir<NRHS, 1, +1>(sl, t, r0, acc);
    if ((sl = advance()) == nullptr) break;
    consume_dir<NRHS, 1, -1>(sl, t, r0, acc);
    if ((sl = advance()) == nullptr) break;
    consume_dir<NRHS, 2, +1>(sl, t, r0, acc);
    if ((sl = advance()) == nullptr) break;
    consume_dir<NRHS, 2, -1>(sl, t, r0, acc);
    if ((sl = advance()) == nullptr) break;
    consume_dir<NRHS, 3, +1>(sl, t, r0, acc);
    if ((sl = advance()) == nullptr) break;
    consume_dir<NRHS, 3, -1>(sl, t, r0, acc);
#pragma unroll
    for (int k = 0; k < 12; ++k)
#pragma unroll
      for (int q = 0; q < 2; ++q) { acc[k].re[q] *= a.c_hop; acc[k].im[q] *= a.c_hop; }
    float m[36];
    const float4* blk = nullptr;
    if constexpr (HAS_SITE) {
      if ((sl = advance()) == nullptr) break;
      blk = reinterpret_cast<const float4*>(sl + (size_t)Sh::TPW * Sh::SP + (size_t)t * kBlockBytes);
      if constexpr (SELF != SELF_NONE) {
        MC<float, 2> s[12];
        lds_spinor<NRHS>(sl, t, r0, 0, s);
        lds_spinor<NRHS>(sl, t, r0, 6, s + 6);
        if constexpr (SELF == SELF_SCALAR) {
#pragma unroll
          for (int k = 0; k < 12; ++k)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              acc[k].re[q] = fmaf(a.self_scalar, s[k].re[q], acc[k].re[q]);
              acc[k].im[q] = fmaf(a.self_scalar, s[k].im[q], acc[k].im[q]);
            }
        } else {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int k = 0; k < 9; ++k) {
              const float4 q = blk[9 * h + k];
              m[4 * k] = q.x; m[4 * k + 1] = q.y; m[4 * k + 2] = q.z; m[4 * k + 3] = q.w;
            }
            MC<float, 2> tt[6];
            block_matvec<float, 2>(m, s + 6 * h, tt);
#pragma unroll
            for (int k = 0; k < 6; ++k)
#pragma unroll
              for (int q = 0; q < 2; ++q) { acc[6 * h + k].re[q] += tt[k].re[q]; acc[6 * h + k].im[q] += tt[k].im[q]; }
          }
        }
      }
    }
    if (site < a.n_target) {
      int p, cb;
      if (a.full) {
        p = site >= a.g.Vh ? 1 : 0;
        cb = site - p * a.g.Vh;
      } else {
        p = a.target_parity;
        cb = site;
      }
      float2* op = a.out + (a.full ? (int64_t)p * a.half_elems : 0) + (int64_t)cb * 12 * NRHS + r0;
      if constexpr (POST == POST_BLOCKINV) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
          for (int k = 0; k < 9; ++k) {
            const float4 q = blk[9 * h + k];
            m[4 * k] = q.x; m[4 * k + 1] = q.y; m[4 * k + 2] = q.z; m[4 * k + 3] = q.w;
          }
          MC<float, 2> tt[6];
          block_matvec<float, 2>(m, acc + 6 * h, tt);
#pragma unroll
          for (int k = 0; k < 6; ++k) mc_store(op + (6 * h + k) * NRHS, tt[k]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          if (POST == POST_SCALAR) {
#pragma unroll
            for (int q = 0; q < 2; ++q) { acc[k].re[q] *= a.post_scalar; acc[k].im[q] *= a.post_scalar; }
          }
          mc_store(op + k * NRHS, acc[k]);
        }
      }
    }
  }
  if (!ok) {
    if (lane == 0 && a.err != nullptr) atomicOr(a.err, 1);
    // the copies still in flight land before the shared memory is released
    const int last = issued < total ? issued : total;
    for (int q = seq + 1; q < last; ++q) mbar_wait_bounded(&bars[q % K], (uint32_t)(q / K) & 1u);
  }
}

}  // namespace ring

// Launch the ring kernel for one (SELF, POST) combination with `warps` warps per CTA
// and `slots` ring slots per warp: a persistent grid of at most (resident CTAs per SM)
// x (SMs) CTAs. cudaErrorInvalidValue if the arguments do not fit (rhs count, site
// tile, missing padded link / block copies, shared memory, unsupported combination).
template <int SELF, int POST, int NRHS, int MAXT, int MINB>
cudaError_t launch_dslash_ring_one(DslashArgs<float> a, int warps, int slots, cudaStream_t stream) {
  if (warps * 32 > MAXT) return cudaErrorInvalidValue;
  auto kern = ring::dslash_ring_kernel<SELF, POST, NRHS, MAXT, MINB>;
  static std::once_flag attr;
  std::call_once(attr, [&] {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  });
  const size_t smem = ring::smem_bytes<NRHS>(warps, slots);
  // resident CTAs per SM of this launch shape (depends on the kernel and the architecture only)
  static std::atomic<int> occ_cache[17][9];
  int occ = occ_cache[warps][slots].load(std::memory_order_relaxed);
  if (occ == 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, warps * 32, smem);
    if (occ < 1) return cudaErrorInvalidValue;
    occ_cache[warps][slots].store(occ, std::memory_order_relaxed);
  }
  constexpr int TPW = ring::Shape<NRHS>::TPW;
  const int64_t tasks = (a.n_target + TPW - 1) / TPW;
  const int64_t need = (tasks + warps - 1) / warps;
  const int64_t cap = (int64_t)(a.num_sms > 0 ? a.num_sms : 1) * occ;
  const int grid = (int)(need < cap ? need : cap);
  a.ring_slots = slots;
  kern<<<grid, warps * 32, smem, stream>>>(a);
  return cudaGetLastError();
}

// Register budgets of the ring kernel: up to 8 warps per CTA with one CTA per SM, or
// up to 7 warps per CTA with two CTAs per SM (<= 146 registers), or up to 16 warps per
// CTA with one CTA per SM (<= 128 registers).
template <int SELF, int POST, int NRHS>
cudaError_t launch_dslash_ring_shape(const DslashArgs<float>& a, int warps, int slots, int ctas_per_sm,
                                     cudaStream_t stream) {
  if (ctas_per_sm == 2) return launch_dslash_ring_one<SELF, POST, NRHS, 224, 2>(a, warps, slots, stream);
  if (warps > 8) return launch_dslash_ring_one<SELF, POST, NRHS, 512, 1>(a, warps, slots, stream);
  return launch_dslash_ring_one<SELF, POST, NRHS, 256, 1>(a, warps, slots, stream);
}

template <int NRHS>
cudaError_t launch_dslash_ring(const DslashArgs<float>& a, int self_mode, int post_mode, int warps, int slots,
                               int ctas_per_sm, cudaStream_t stream) {
  if (a.lay.nrhs != NRHS || a.lay.log_s != 0 || a.links_aos == nullptr) return cudaErrorInvalidValue;
  if (warps < 1 || warps > 16 || slots < 1 || slots > 8 || ctas_per_sm < 1 || ctas_per_sm > 2)
    return cudaErrorInvalidValue;
  if ((size_t)ctas_per_sm * ring::smem_bytes<NRHS>(warps, slots) > 227 * 1024) return cudaErrorInvalidValue;
  if ((self_mode == SELF_BLOCK && a.blocks_aos == nullptr) ||
      (post_mode == POST_BLOCKINV && a.blocks_inv_aos == nullptr))
    return cudaErrorInvalidValue;
  if (self_mode == SELF_SCALAR && post_mode == POST_NONE)
    return launch_dslash_ring_shape<SELF_SCALAR, POST_NONE, NRHS>(a, warps, slots, ctas_per_sm, stream);
  if (self_mode == SELF_BLOCK && post_mode == POST_NONE)
    return launch_dslash_ring_shape<SELF_BLOCK, POST_NONE, NRHS>(a, warps, slots, ctas_per_sm, stream);
  if (self_mode == SELF_NONE && post_mode == POST_SCALAR)
    return launch_dslash_ring_shape<SELF_NONE, POST_SCALAR, NRHS>(a, warps, slots, ctas_per_sm, stream);
  if (self_mode == SELF_NONE && post_mode == POST_BLOCKINV)
    return launch_dslash_ring_shape<SELF_NONE, POST_BLOCKINV, NRHS>(a, warps, slots, ctas_per_sm, stream);
  return cudaErrorInvalidValue;
}

#define LQCD_DSLASH_RING_TU(NRHS) \
  template cudaError_t launch_dslash_ring<NRHS>(const DslashArgs<float>&, int, int, int, int, int, cudaStream_t);

}  // namespace lqcd
