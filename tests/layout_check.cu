// Host-side check of the row-gather shared-memory layout (tests/test_layout_cpu.py).
//
// For every precision, the assembly and the time-step layouts, block sizes
// R in {32, 64, 96, 128}, row lengths W up to 32 and several entry and step
// counts, the regions the kernels carve out of one block's shared memory must
// be 16-byte aligned (asynchronous 16-byte copies land there) and must not
// overlap, and the aliases the kernels rely on must fit:
//   col (4 bytes per CSR entry) inside nb1;
//   the second half of each staged 32-byte record (mixed: one 16-byte half,
//   FP64: two 16-byte planes) inside the slot's accumulator bytes;
//   the write-out's staging of the block's entries inside nb0;
//   the time step's one accumulator per slot at the 16-byte record stride.
// Prints one summary line; exit code 0 when every case holds.
#include <cstdio>

#include "../paper_2111_05651_gb300/csrc/nsi_internal.cuh"

int main() {
  long cases = 0, bad = 0;
  auto check = [&](bool ok, const char* what, int prec, bool step, int R, int W, int L, int S) {
    if (!ok && bad++ < 10)
      std::printf("FAIL %s (precision %d, step %d, R %d, W %d, L %d, S %d)\n", what, prec, (int)step, R, W, L, S);
  };
  for (int prec : {NSI_FP64, NSI_MIXED_F32_ACC64, NSI_MIXED_F32_ACC32})
    for (bool step : {false, true})
      for (int R : {32, 64, 96, 128})
        for (int W = 1; W <= 32; ++W)
          for (int Lq : {0, 1, 2, 3, 4}) {
            const int N = R * W, L = N * Lq / 4;
            for (int S : {0, 1, 7, 100, 4095}) {
              const nsi::GatherSmem g = nsi::gather_smem(prec, R, W, L, S, step);
              ++cases;
              const size_t tb = g.tb, n = g.N();
              check(g.nb1() % 16 == 0 && g.acc() % 16 == 0 && g.walk() % 16 == 0 && g.stat() % 16 == 0 &&
                        g.total() % 16 == 0,
                    "16-byte alignment", prec, step, R, W, L, S);
              check(g.nb0() + 4 * tb * n <= g.nb1() && g.nb1() + 2 * tb * n <= g.acc() &&
                        g.acc() + (size_t)g.ab * n <= g.walk() && g.walk() + (size_t)S + 8 <= g.stat() &&
                        g.stat() + (size_t)g.xs * L <= g.total(),
                    "regions in order without overlap", prec, step, R, W, L, S);
              check((size_t)4 * L <= 2 * tb * n, "column indices inside nb1", prec, step, R, W, L, S);
              const size_t half = prec == NSI_FP64 ? 32 : 16;  // bytes of staged record halves per slot
              check(half <= (size_t)g.ab, "staged record halves inside the accumulators", prec, step, R, W, L, S);
              if (!step) {
                check(g.stage_fits(), "write-out staging inside nb0", prec, step, R, W, L, S);
                if (prec == NSI_MIXED_F32_ACC64) {
                  // A pairs and G_x, G_y in nb0; G_z in the half of nb1 past the column indices
                  check((size_t)16 * L <= 4 * tb * n, "pair staging inside nb0", prec, step, R, W, L, S);
                  check(g.nb1() + 4 * n + 4 * (size_t)L <= g.acc() && (size_t)4 * L <= 4 * n,
                        "G_z staging inside nb1 past the column indices", prec, step, R, W, L, S);
                }
              } else {
                check((size_t)g.ob * L <= 4 * tb * n && (size_t)8 * L <= 4 * tb * n, "step staging inside nb0", prec,
                      step, R, W, L, S);
                check((size_t)g.ab >= 16, "one accumulator per slot at the 16-byte stride", prec, step, R, W, L, S);
                check(g.xs == g.ob, "A_static slice of one output value per entry", prec, step, R, W, L, S);
              }
            }
          }
  std::printf("cases=%ld failures=%ld\n", cases, bad);
  return bad == 0 ? 0 : 1;
}
