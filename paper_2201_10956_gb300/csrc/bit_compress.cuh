// Bit extraction for the sample compaction of the tensor scan, usable from host and device code
// (the host tests check it against a plain bit loop).
#pragma once

#include <cstdint>

namespace epi3 {

// Bit extraction ("compress", Hacker's Delight sec. 7-4): the bits of x at the set positions
// of m, packed to the low end in order.  The five move masks depend on m only and are computed
// once per mask word by cmp_masks.
__host__ __device__ __forceinline__ void cmp_masks(uint32_t m, uint32_t* mv) {
    uint32_t mk = ~m << 1;
    for (int t = 0; t < 5; ++t) {
        uint32_t mp = mk ^ (mk << 1);
        mp ^= mp << 2;
        mp ^= mp << 4;
        mp ^= mp << 8;
        mp ^= mp << 16;
        const uint32_t v = mp & m;
        m = (m ^ v) | (v >> (1u << t));
        mk &= ~mp;
        mv[t] = v;
    }
}
__host__ __device__ __forceinline__ uint32_t cmp_bits(uint32_t x, uint32_t m, const uint32_t* mv) {
    x &= m;
    for (int t = 0; t < 5; ++t) {
        const uint32_t u = x & mv[t];
        x = (x ^ u) | (u >> (1u << t));
    }
    return x;
}


}  // namespace epi3
