// rng.cuh -- counter-based generators of the workloads, device side.
//
// Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As Easy
// as 1, 2, 3" (SC'11), Sec. 4.2 -- ten rounds of two 32x32->64 multiplies by
// fixed odd constants whose high halves are xored with the other two words and
// the round key, followed by a word permutation; the key advances by Weyl
// increments between rounds.
// SplitMix64: Steele, Lea, Flood (OOPSLA'14) -- add the golden gamma, then the
// xor-shift/multiply finaliser of the JDK 8 SplittableRandom.
#pragma once
#include <cstdint>

__device__ __forceinline__ uint32_t dsoa_philox_w0(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                                                   uint32_t c3) {
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo_a = 0xD2511F53u * c0, hi_a = __umulhi(0xD2511F53u, c0);
        const uint32_t lo_b = 0xCD9E8D57u * c2, hi_b = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi_b ^ c1 ^ k0, n2 = hi_a ^ c3 ^ k1;
        c0 = n0; c1 = lo_b; c2 = n2; c3 = lo_a;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    return c0;
}

__device__ __forceinline__ uint64_t dsoa_splitmix(uint64_t s) {
    uint64_t z = s + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t dsoa_sm2(uint64_t a, uint64_t b) { return dsoa_splitmix(dsoa_splitmix(a) ^ b); }
__device__ __forceinline__ uint64_t dsoa_sm3(uint64_t a, uint64_t b, uint64_t c) {
    return dsoa_splitmix(dsoa_sm2(a, b) ^ c);
}
