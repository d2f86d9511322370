// Host-only check of the streaming Gram-Schmidt tile plans (no kernel is launched): for every
// plan make_plan can return, the bulk copies of a stage are 16-byte aligned in size and offset
// (tail tiles included), the stage layout and the reduction scratch fit the shared-memory budget
// of the instance, the mbarrier header fits its 128 bytes and a stage's transaction count fits
// an mbarrier. Exit status 0 when every plan passes.
#include <cstdio>

#include "../paper_2601_05816_gb300/csrc/gs_stream.cuh"

using namespace lqcd::gss;

static int bad = 0;
#define CHECK(cond, ...)                                   \
  do {                                                     \
    if (!(cond)) {                                         \
      if (bad < 20) {                                      \
        std::printf("FAIL %s: ", #cond);                   \
        std::printf(__VA_ARGS__);                          \
        std::printf("\n");                                 \
      }                                                    \
      ++bad;                                               \
    }                                                      \
  } while (0)

int main() {
  long plans = 0;
  const int elems[2] = {4, 8};  // BF16 pair, FP32 complex
  for (int eb : elems)
    for (int nrhs = 1; nrhs <= 64; ++nrhs)
      for (int epl = 1; epl <= 2; ++epl) {
        if (nrhs % epl != 0 || nrhs / epl > 32) continue;
        for (int nvec = 1; nvec <= 32; ++nvec) {
          const int nv = nvec <= 8 ? 8 : (nvec <= 16 ? 16 : (nvec <= 24 ? 24 : 32));
          for (int update = 0; update <= 1; ++update) {
            const Plan p = make_plan(nrhs, nvec, nv, epl, eb, update != 0);
            if (!p.ok) continue;
            ++plans;
            const bool two = two_ctas(nv, epl);
            const size_t budget = two ? 112 * 1024 : 225 * 1024;
            const size_t red_one = (size_t)kConsumers * epl * 32 * 16;
            const long TR = p.TR;
            CHECK(p.lpr * epl == nrhs && p.H == 32 / p.lpr, "nrhs %d epl %d", nrhs, epl);
            CHECK(TR == (long)kConsumers * p.H * p.J, "nrhs %d TR %ld", nrhs, TR);
            // bulk copies: basis tiles and the FP32 w tile, 16-byte sizes and offsets
            CHECK((TR * nrhs * eb) % 16 == 0, "basis tile bytes, nrhs %d TR %ld eb %d", nrhs, TR, eb);
            CHECK((TR * nrhs * 8) % 16 == 0, "w tile bytes, nrhs %d TR %ld", nrhs, TR);
            CHECK(p.vt_bytes == (uint32_t)(TR * nrhs * eb) && p.vt_bytes % 16 == 0, "vt_bytes");
            CHECK(p.stage_bytes >= (uint64_t)nvec * p.vt_bytes + TR * nrhs * 8 && p.stage_bytes % 128 == 0,
                  "stage bytes, nrhs %d nvec %d", nrhs, nvec);
            // a tail tile of any length that keeps n * eb a multiple of 16 also has 16-byte sizes
            for (long Q = 1; Q <= 3 * TR; ++Q) {
              if ((Q * nrhs * eb) % 16 != 0) continue;
              const long rows = Q % TR == 0 ? TR : Q % TR;
              CHECK((rows * nrhs * eb) % 16 == 0 && (rows * nrhs * 8) % 16 == 0, "tail Q %ld nrhs %d", Q, nrhs);
            }
            // shared memory: header (2 S mbarriers + flag) in 128 bytes, coefficients, stages
            CHECK(p.S >= 2 && 16 * p.S + 4 <= 128, "stages %d", p.S);
            CHECK(p.coef_off == 128 && p.stage_off % 128 == 0, "offsets");
            CHECK(p.stage_off >= 128 + (update ? (size_t)nvec * nrhs * 8 : 0), "coefficients, nvec %d", nvec);
            const size_t st = (size_t)p.S * p.stage_bytes > red_one ? (size_t)p.S * p.stage_bytes : red_one;
            CHECK(p.smem == p.stage_off + st && p.smem <= budget, "smem %zu budget %zu", p.smem, budget);
            CHECK(p.red_vecs >= 1 && p.red_vecs <= nvec && (size_t)p.red_vecs * red_one <= st, "red_vecs %d",
                  p.red_vecs);
            // one stage's transaction count must fit an mbarrier's (2^20 - 1 bytes)
            CHECK((uint64_t)nvec * p.vt_bytes + TR * nrhs * 8 < (1u << 20), "tx count");
            CHECK(p.ctas_per_sm == (two ? 2 : 1), "ctas per SM");
          }
        }
      }
  std::printf("%ld plans checked, %d failures\n", plans, bad);
  return bad == 0 && plans > 0 ? 0 : 1;
}
