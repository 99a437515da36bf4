// Host check of the compaction's bit extraction (cmp_masks + cmp_bits) against a plain loop
// that keeps the bits of x at the set positions of m, in order, packed to the low end.
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include "../../paper_2201_10956_gb300/csrc/bit_compress.cuh"
static uint32_t rnd() { return ((uint32_t)rand() << 16) ^ (uint32_t)rand(); }
int main() {
  srand(7);
  for (int trial = 0; trial < 200000; ++trial) {
    uint32_t x = rnd(), m = rnd();
    if (trial % 7 == 0) m = 0xFFFFFFFFu;
    if (trial % 11 == 0) m = 0u;
    if (trial % 13 == 0) m &= rnd() & rnd();
    uint32_t want = 0; int k = 0;
    for (int b = 0; b < 32; ++b)
      if ((m >> b) & 1u) { want |= ((x >> b) & 1u) << k; ++k; }
    uint32_t mv[5];
    epi3::cmp_masks(m, mv);
    const uint32_t got = epi3::cmp_bits(x, m, mv);
    if (got != want) { printf("MISMATCH x=%08x m=%08x got=%08x want=%08x\n", x, m, got, want); return 1; }
  }
  printf("bit compress ok\n");
  return 0;
}
