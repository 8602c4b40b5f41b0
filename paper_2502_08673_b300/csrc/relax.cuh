// Arithmetic of the relaxation shared by the step kernels (tiled and shared-memory
// resident), so that both compute every value with the same operations in the same
// order: the embedding (Eq. 5), the gates' bilinear forms (Table 1), the Adam bias
// corrections and the input update (Eq. 9 / Adam).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "device.hpp"

namespace sat {

__device__ __forceinline__ float sigmoidf_(float v) { return 1.0f / (1.0f + expf(-v)); }

// Bilinear coefficients (k0, k1, k2, k3) of gate code gop = op | neg0 << 2 |
// neg1 << 3, with a' = n0 + s0 a and b' = n1 + s1 b (s = 1 - 2 n):
//   AND a'b':         (n0 n1,             s0 n1,         n0 s1,         s0 s1)
//   OR a'+b'-a'b':    (n0 + n1 - n0 n1,   s0 (1 - n1),   s1 (1 - n0),  -s0 s1)
//   XOR a'+b'-2a'b':  (n0 + n1 - 2 n0 n1, s0 (1 - 2 n1), s1 (1 - 2 n0), -2 s0 s1)
__device__ __forceinline__ float4 gate_coeffs(uint32_t gop) {
    const float n0 = (float)((gop >> 2) & 1u), n1 = (float)((gop >> 3) & 1u);
    const float s0 = 1.0f - 2.0f * n0, s1 = 1.0f - 2.0f * n1;
    switch (gop & 3u) {
    case 0: return make_float4(n0 * n1, s0 * n1, n0 * s1, s0 * s1);
    case 1: return make_float4(n0 + n1 - n0 * n1, s0 * (1.0f - n1), s1 * (1.0f - n0), -s0 * s1);
    default: return make_float4(n0 + n1 - 2.0f * n0 * n1, s0 * (1.0f - 2.0f * n1), s1 * (1.0f - 2.0f * n0),
                                -2.0f * s0 * s1);
    }
}

// (The tiled step kernel evaluates the same three fmas on two samples at a time with the
// packed FP32 fma, which rounds each element exactly as fmaf does.)
__device__ __forceinline__ float gate_apply(const float4& k, float a, float b) {
    return fmaf(fmaf(k.w, a, k.z), b, fmaf(k.y, a, k.x));
}

// Adam bias corrections at step t >= 1 (PyTorch: step_size = lr / (1 - b1^t),
// sqrt(1 - b2^t)) in FP32: 1 - b^t = -expm1(t log1p(b - 1)).  b - 1 is exact in
// FP32 for b in [1/2, 2], so both corrections keep ~1e-7 relative accuracy even
// where b^t is within 1e-3 of 1 (b2 = 0.999 at t = 1).
__device__ __forceinline__ void adam_bias(const OptParams& o, int t, float& step_size, float& bc2s) {
    const float tf = (float)t;
    step_size = o.lr / -expm1f(tf * log1pf(o.b1 - 1.0f));
    bc2s = sqrtf(-expm1f(tf * log1pf(o.b2 - 1.0f)));
}

// dL/dV = Pbar * P (1 - P) for one sample with P = sigmoid(vv) given, then GD (Eq. 9) or
// Adam (PyTorch's formulation, no weight decay) on V, m, v at element r.  Returns the new
// V (vv when only the gradient is stored).
template <bool UPDATE>
__device__ __forceinline__ float input_update_p(const OptParams& o, float* V, float* m, float* v, float* gV, int64_t r,
                                                float vv, float P, float pbar, float mm, float ss, float step_size,
                                                float bc2s) {
    const float g = pbar * P * (1.0f - P);
    if (!UPDATE) {
        gV[r] = g;
        return vv;
    } else if (o.opt == 1) {
        const float nv = fmaf(-o.lr, g, vv);
        V[r] = nv;
        return nv;
    } else {
        const float m1 = fmaf(1.0f - o.b1, g - mm, mm);
        const float v1 = fmaf(o.b2, ss, (1.0f - o.b2) * g * g);
        m[r] = m1;
        v[r] = v1;
        const float nv = vv - step_size * (m1 / (sqrtf(v1) / bc2s + o.eps));
        V[r] = nv;
        return nv;
    }
}

// The same with P computed here.
template <bool UPDATE>
__device__ __forceinline__ float input_update(const OptParams& o, float* V, float* m, float* v, float* gV, int64_t r,
                                              float vv, float pbar, float mm, float ss, float step_size, float bc2s) {
    return input_update_p<UPDATE>(o, V, m, v, gV, r, vv, sigmoidf_(vv), pbar, mm, ss, step_size, bc2s);
}

// Partial sums of the per-sample loss: outputs j = w, w + n, w + 2n, ... go to partial w
// (n = 20 for FP32 activations, 24 for 16-bit ones), and the partials are added in order.
template <typename T>
__host__ __device__ constexpr int loss_partials() { return sizeof(T) == 4 ? 20 : 24; }

}  // namespace sat
