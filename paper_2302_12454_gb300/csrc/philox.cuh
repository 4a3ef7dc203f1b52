// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel
// random numbers: as easy as 1, 2, 3", SC'11), device side.  The paper's
// noise r_i(t) (Eq. 2a, Eq. 6a) is a random +-1 per spin and cycle; its
// generator is not specified, so this library draws it from Philox keyed by
// the anneal seed.  Spins are grouped in 32-spin words w = i / 32; word w
// takes output word (w / 4) % 4 of the call with counter
// (4 (w / 16) + w % 4, replica k, trial, cycle t), so one call covers the
// four words w, w + 4, w + 8, w + 12 of a 16-word group.
#pragma once
#include <cstdint>

namespace ssqa {

struct Philox4 {
    uint32_t x[4];
};

// Ten rounds of the Philox-4x32 S-box: multiply two words by the published
// constants, cross the high halves with the other words and the round key,
// then advance the key by the Weyl increments.
__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        const uint32_t p0_lo = m0 * c0, p0_hi = __umulhi(m0, c0);
        const uint32_t p1_lo = m1 * c2, p1_hi = __umulhi(m1, c2);
        const uint32_t n0 = p1_hi ^ c1 ^ k0;
        const uint32_t n2 = p0_hi ^ c3 ^ k1;
        c0 = n0;
        c1 = p1_lo;
        c2 = n2;
        c3 = p0_lo;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    Philox4 o;
    o.x[0] = c0;
    o.x[1] = c1;
    o.x[2] = c2;
    o.x[3] = c3;
    return o;
}

// Position of spin i's bit inside its 32-bit word.  Pairs of spins (2j,
// 2j+1) of a 32-spin group sit at bits 15-j and 31-j, so `(w << j) &
// 0x80008000` moves both into the sign bits of a packed half2.  A set bit
// means r = -1 (noise) or sigma = -1 (initial spin).
__device__ __forceinline__ uint32_t spin_bit_pos(uint32_t i) {
    const uint32_t e = i & 31u;
    return (e & 1u) ? (31u - (e >> 1)) : (15u - (e >> 1));
}

// Counter word of the Philox call serving 32-spin word `w`, and the output
// word of that call it takes.
__device__ __forceinline__ uint32_t noise_ctr(uint32_t w) { return 4u * (w >> 4) + (w & 3u); }
__device__ __forceinline__ uint32_t noise_out(uint32_t w) { return (w >> 2) & 3u; }

__device__ __forceinline__ uint32_t noise_word(uint64_t seed, uint32_t i, uint32_t k, uint32_t trial,
                                               uint32_t t) {
    const uint32_t wd = i >> 5;
    const Philox4 o = philox4x32_10(noise_ctr(wd), k, trial, t, uint32_t(seed), uint32_t(seed >> 32));
    const uint32_t w = noise_out(wd);
    return w == 0 ? o.x[0] : (w == 1 ? o.x[1] : (w == 2 ? o.x[2] : o.x[3]));
}

}  // namespace ssqa
