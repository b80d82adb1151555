// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw, SC'11), device side.
// Round: (c0,c1,c2,c3),(k0,k1) -> (hi(B*c2)^c1^k0, lo(B*c2), hi(A*c0)^c3^k1, lo(A*c0)),
// A = 0xD2511F53, B = 0xCD9E8D57; key bumped by (0x9E3779B9, 0xBB67AE85) between rounds.
#pragma once

#include <stdint.h>

namespace rbsog {

struct U4 {
    uint32_t x, y, z, w;
};

__host__ __device__ inline U4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        unsigned long long pa = (unsigned long long)0xD2511F53u * c0;
        unsigned long long pb = (unsigned long long)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(pb >> 32) ^ c1 ^ k0;
        uint32_t n2 = (uint32_t)(pa >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)pb;
        c3 = (uint32_t)pa;
        c0 = n0;
        c2 = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return U4{c0, c1, c2, c3};
}

// uniform double in [0,1): the 53-bit integer (a >> 11, b) times 2^-53
__host__ __device__ inline double u53_of(uint32_t a, uint32_t b) {
    unsigned long long v = ((unsigned long long)(a >> 11) << 32) | (unsigned long long)b;
    return (double)v * 1.1102230246251565404e-16;
}

}  // namespace rbsog
