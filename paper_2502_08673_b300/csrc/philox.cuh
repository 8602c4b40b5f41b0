// Counter-based normal draws shared by the initialisation kernels (sm_103a).
#pragma once

#include <cstdint>

namespace sat {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ uint4 philox4x32_10(uint4 ctr, uint2 key) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const uint32_t hi0 = __umulhi(M0, ctr.x), lo0 = M0 * ctr.x;
        const uint32_t hi1 = __umulhi(M1, ctr.z), lo1 = M1 * ctr.z;
        ctr = make_uint4(hi1 ^ ctr.y ^ key.x, lo1, hi0 ^ ctr.w ^ key.y, lo0);
        key.x += W0;
        key.y += W1;
    }
    return ctr;
}

// Box-Muller from two Philox words: u1 = ((first >> 8) + 1) / 2^24 in (0, 1] gives the
// radius sqrt(-2 ln u1), u2 = (second >> 8) / 2^24 the angle 2 pi u2 (sine and cosine).
__device__ __forceinline__ float bm_radius(uint32_t first) {
    const float u1 = (float)((first >> 8) + 1u) * (1.0f / 16777216.0f);
    return sqrtf(-2.0f * logf(u1));
}
__device__ __forceinline__ void bm_angle(uint32_t second, float* sn, float* cs) {
    const float u2 = (float)(second >> 8) * (1.0f / 16777216.0f);
    sincospif(2.0f * u2, sn, cs);
}

// Four standard normals of input row r for samples 4c .. 4c + 3: the Philox4x32-10 block at
// counter (c, r, round, 0) gives two Box-Muller pairs, (cos, sin) of words (x, y) and of
// words (z, w).
__device__ __forceinline__ float4 normal4(uint32_t c, uint32_t r, uint32_t round, uint2 key) {
    const uint4 o = philox4x32_10(make_uint4(c, r, round, 0u), key);
    float4 z;
    {
        const float rad = bm_radius(o.x);
        float sn, cs;
        bm_angle(o.y, &sn, &cs);
        z.x = rad * cs;
        z.y = rad * sn;
    }
    {
        const float rad = bm_radius(o.z);
        float sn, cs;
        bm_angle(o.w, &sn, &cs);
        z.z = rad * cs;
        z.w = rad * sn;
    }
    return z;
}

// Signs (-1, 0, +1) of the cosine and sine of the Box-Muller angle, read off its place on the
// grid: the angle is pi x with x = k / 2^23, k = second >> 8, and cos(pi x) > 0 on [0, 1/2) and
// (3/2, 2), = 0 at 1/2 and 3/2, sin(pi x) > 0 on (0, 1), = 0 at 0 and 1.  sincospif's results
// have these signs at every one of the 2^24 grid points (checked by sat_diag_angle_signs).
__device__ __forceinline__ void bm_angle_signs(uint32_t second, int* cs, int* sn) {
    const uint32_t k = second >> 8;
    *cs = k < 0x400000u ? 1 : k == 0x400000u ? 0 : k < 0xC00000u ? -1 : k == 0xC00000u ? 0 : 1;
    *sn = k == 0u ? 0 : k < 0x800000u ? 1 : k == 0x800000u ? 0 : -1;
}

// The threshold bits [scale * z_k > 0] of the same four normals (bit k: sample 4c + k),
// without forming them, for |scale| >= 2^-60 (positive = scale > 0): the radius is 0 exactly
// when u1 = 1 (first >> 8 = 2^24 - 1; then z = +-0) and positive otherwise, and scale * radius
// * (sine or cosine) cannot underflow to 0 (radius >= 3.4e-4, a nonzero sine or cosine of the
// angle grid >= 3.7e-7), so the sign is that of scale times the sine or cosine: no logarithm,
// square root or sine.
constexpr float BITS_MIN_SCALE = 8.6736174e-19f;  // 2^-60
__device__ __forceinline__ uint32_t normal4_bits(uint32_t c, uint32_t r, uint32_t round, uint2 key, bool positive) {
    const uint4 o = philox4x32_10(make_uint4(c, r, round, 0u), key);
    const int want = positive ? 1 : -1;
    uint32_t bits = 0u;
    int cs, sn;
    bm_angle_signs(o.y, &cs, &sn);
    if ((o.x >> 8) != 0xFFFFFFu) bits |= (cs == want ? 1u : 0u) | (sn == want ? 2u : 0u);
    bm_angle_signs(o.w, &cs, &sn);
    if ((o.z >> 8) != 0xFFFFFFu) bits |= (cs == want ? 4u : 0u) | (sn == want ? 8u : 0u);
    return bits;
}
// The same bits for any scale, from the normals themselves.
__device__ __forceinline__ uint32_t normal4_bits_formed(uint32_t c, uint32_t r, uint32_t round, uint2 key, float scale) {
    const float4 z = normal4(c, r, round, key);
    return (scale * z.x > 0.0f ? 1u : 0u) | (scale * z.y > 0.0f ? 2u : 0u) | (scale * z.z > 0.0f ? 4u : 0u) |
           (scale * z.w > 0.0f ? 8u : 0u);
}

}  // namespace sat
