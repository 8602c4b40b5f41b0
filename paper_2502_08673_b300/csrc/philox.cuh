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

// Four standard normals of input row r for samples 4c .. 4c + 3: the Philox4x32-10 block at
// counter (c, r, round, 0) gives two Box-Muller pairs, (cos, sin) of words (x, y) and of
// words (z, w), with u1 = ((first >> 8) + 1) / 2^24 and u2 = (second >> 8) / 2^24.
__device__ __forceinline__ float4 normal4(uint32_t c, uint32_t r, uint32_t round, uint2 key) {
    const uint4 o = philox4x32_10(make_uint4(c, r, round, 0u), key);
    float4 z;
    {
        const float u1 = (float)((o.x >> 8) + 1u) * (1.0f / 16777216.0f);
        const float u2 = (float)(o.y >> 8) * (1.0f / 16777216.0f);
        const float rad = sqrtf(-2.0f * logf(u1));
        float sn, cs;
        sincospif(2.0f * u2, &sn, &cs);
        z.x = rad * cs;
        z.y = rad * sn;
    }
    {
        const float u1 = (float)((o.z >> 8) + 1u) * (1.0f / 16777216.0f);
        const float u2 = (float)(o.w >> 8) * (1.0f / 16777216.0f);
        const float rad = sqrtf(-2.0f * logf(u1));
        float sn, cs;
        sincospif(2.0f * u2, &sn, &cs);
        z.z = rad * cs;
        z.w = rad * sn;
    }
    return z;
}

}  // namespace sat
