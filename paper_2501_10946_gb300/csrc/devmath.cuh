// FP32 phase and summation helpers shared by the structure-factor and gather kernels.
#pragma once

#include <stdint.h>

namespace rbsog {

constexpr float kTwoPiOver2p32 = 1.4629180792671596e-09f;   // 2 pi / 2^32

// exp(i 2 pi th / 2^32) for an exact integer phase th (turns x 2^32), up to a sign.
// Half-turn reduction: th = r + q 2^31 with r in [-2^30, 2^30), so the result is
// (-1)^q exp(i 2 pi r / 2^32); the sign (-1)^q comes back as a float sign-bit mask.
// Besides halving the argument range, this makes the remaining errors of the float
// scaling and of the special-function unit enter with a zero-mean factor (-1)^q, so
// they do not add up coherently over many particles.
__device__ __forceinline__ uint32_t half_turn_sincos(uint32_t th, float &sn, float &cs) {
    const uint32_t sgn = (th ^ (th << 1)) & 0x80000000u;   // |phase| >= 1/4 turn
    const float x = (float)(int)(th ^ sgn) * kTwoPiOver2p32;
    __sincosf(x, &sn, &cs);
    return sgn;
}

__device__ __forceinline__ float flip(float v, uint32_t sgn) { return __uint_as_float(__float_as_uint(v) ^ sgn); }

__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
}

}  // namespace rbsog
