// sl_fastnormal.cuh -- the Philox4x32-10 / Box-Muller normals of normal4 evaluated on the
// special-function unit: the same counter words and pairs, with the fast logarithm,
// sine/cosine and square root (errors of a few 1e-7 relative to the normal's scale).
#pragma once

#include "sl_internal.cuh"

namespace sl {

// Square root on the special-function unit (relative error near one ulp, the size of the
// other FP32 roundings of the kernels that use it).
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// -2 log u for u in (0, 1): the fast base-2 logarithm (absolute error near 2^-22), except within
// 2^-7 of 1, where -log(1 - t) = t + t^2/2 + t^3/3 + t^4/4 + O(t^5) in t = 1 - u (exact in FP32)
// keeps the small result's relative accuracy (the series' remainder is below 1e-9 of it).
__device__ __forceinline__ float minus_2log(float u) {
    const float t = 1.0f - u;
    float lg;
    asm("lg2.approx.f32 %0, %1;" : "=f"(lg) : "f"(u));
    const float ser = 2.0f * t * fmaf(t, fmaf(t, fmaf(t, 0.25f, 0.333333333f), 0.5f), 1.0f);
    return t < 0.0078125f ? ser : -1.38629436f * lg;
}

// The uniform ((w >> 9) + 1/2) 2^-23 of word_to_uniform without an integer-to-float conversion:
// 1 + (w >> 9) 2^-23 is the float with those mantissa bits, and subtracting 1 - 2^-24 (exact in
// FP32) is exact by Sterbenz's lemma, so it gives word_to_uniform's value bit for bit.
constexpr float kOneMinusHalfUlp = 0.99999994039535522f;   // 1 - 2^-24
constexpr float kTwoPi = 6.28318530717958648f;
constexpr float kTwoPiHalfUlp = 3.74507028e-07f;            // 2 pi 2^-24
__device__ __forceinline__ float uniform_bits(uint32_t w) { return __uint_as_float(0x3F800000u | (w >> 9)); }

// Philox4x32-10 with its ten round keys computed once: a kernel that draws many blocks from one
// seed keeps them (uniform across the launch) instead of adding the Weyl increments in every
// call; the words are those of philox4x32_10.
struct PhiloxKeys {
    uint32_t k0[10], k1[10];
};
__device__ __forceinline__ PhiloxKeys philox_keys(uint64_t seed) {
    PhiloxKeys K;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        K.k0[r] = static_cast<uint32_t>(seed) + static_cast<uint32_t>(r) * 0x9E3779B9u;
        K.k1[r] = static_cast<uint32_t>(seed >> 32) + static_cast<uint32_t>(r) * 0xBB67AE85u;
    }
    return K;
}
__device__ __forceinline__ uint4 philox4x32_10_keyed(uint4 c, const PhiloxKeys& K) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ K.k0[r], lo1, hi0 ^ c.w ^ K.k1[r], lo0);
    }
    return c;
}

// Normals 4*block .. 4*block+3 for the issue-bound kernels (the EM stage, the 7L-CDC
// paths, the tensor-core sampler): the same Philox4x32-10 words and Box-Muller pairs as
// normal4 (radius sqrt(-2 log u0), angle 2 pi u1; (cos, sin)), with the fast logarithm
// (minus_2log), the fast sine/cosine (absolute error about 2^-21 on [-pi, pi], so the angle is
// taken as 2 pi (u1 - 1/2) and both results negated) and the approximate square root:
// about 25 instructions fewer per pair than normal4.
__device__ __forceinline__ float4 normal4_fast_keyed(const PhiloxKeys& K, uint32_t tag, uint32_t set,
                                                     uint32_t path, uint32_t block) {
    const uint4 w = philox4x32_10_keyed(make_uint4(block, path, set, tag), K);
    const float r0 = sqrt_approx(minus_2log(uniform_bits(w.x) - kOneMinusHalfUlp));
    const float r1 = sqrt_approx(minus_2log(uniform_bits(w.z) - kOneMinusHalfUlp));
    float s0, c0, s1, c1;
    // angle 2 pi (u - 1/2) = 2 pi ((1 + m 2^-23) - 3/2) + 2 pi 2^-24, the difference exact
    __sincosf(fmaf(kTwoPi, uniform_bits(w.y) - 1.5f, kTwoPiHalfUlp), &s0, &c0);
    __sincosf(fmaf(kTwoPi, uniform_bits(w.w) - 1.5f, kTwoPiHalfUlp), &s1, &c1);
    return make_float4(-r0 * c0, -r0 * s0, -r1 * c1, -r1 * s1);
}
__device__ __forceinline__ float4 normal4_fast(uint64_t seed, uint32_t tag, uint32_t set, uint32_t path,
                                               uint32_t block) {
    return normal4_fast_keyed(philox_keys(seed), tag, set, path, block);
}

}  // namespace sl
