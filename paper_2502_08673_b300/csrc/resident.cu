// Shared-memory resident step kernel: the fused hot loop (forward, loss, adjoint,
// update; Eqs. 5-9) for circuits whose whole per-sample state fits in one CTA's
// shared memory.  A CTA serves 32 samples, one per lane; its warps divide each
// level's gates (forward) and nodes (adjoint) and meet at __syncthreads between
// levels.  Activations, adjoints and the inputs' V, m, v stay in shared memory
// for all the steps of the launch, so the only device-memory traffic is reading
// and writing V, m, v once and the loss.  The arithmetic is that of the tiled
// kernel (relax.cuh; edges summed in fan-out CSR order; the loss in the tiled
// kernel's partial order), so both give bit-identical results.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>

#include "device.hpp"
#include "relax.cuh"

namespace sat {
namespace {

constexpr int RES_MAX_WARPS = 32;  // warps per CTA for the widest levels

// A CTA serves 32 x SPL samples: lane j holds samples SPL j .. SPL j + SPL - 1, adjacent
// in every shared-memory row, so one (vector) load or store moves a lane's samples.
template <int SPL>
constexpr int res_lanes() { return 32 * SPL; }

// A lane's SPL consecutive values of one row, as FP32.
template <typename T, int SPL>
__device__ __forceinline__ void lane_ld(const T* p, float (&x)[SPL]) {
    if constexpr (SPL == 1) {
        if constexpr (sizeof(T) == 4) x[0] = *reinterpret_cast<const float*>(p);
        else if constexpr (std::is_same<T, __nv_bfloat16>::value) x[0] = __bfloat162float(*p);
        else x[0] = __half2float(*p);
    } else {
        float2 f;
        if constexpr (sizeof(T) == 4) f = *reinterpret_cast<const float2*>(p);
        else if constexpr (std::is_same<T, __nv_bfloat16>::value)
            f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
        else f = __half22float2(*reinterpret_cast<const __half2*>(p));
        x[0] = f.x;
        x[1] = f.y;
    }
}
template <typename T, int SPL>
__device__ __forceinline__ void lane_st(T* p, const float (&x)[SPL]) {
    if constexpr (SPL == 1) {
        if constexpr (sizeof(T) == 4) *reinterpret_cast<float*>(p) = x[0];
        else if constexpr (std::is_same<T, __nv_bfloat16>::value) *p = __float2bfloat16_rn(x[0]);
        else *p = __float2half_rn(x[0]);
    } else {
        if constexpr (sizeof(T) == 4) *reinterpret_cast<float2*>(p) = make_float2(x[0], x[1]);
        else if constexpr (std::is_same<T, __nv_bfloat16>::value)
            *reinterpret_cast<__nv_bfloat162*>(p) = __float22bfloat162_rn(make_float2(x[0], x[1]));
        else *reinterpret_cast<__half2*>(p) = __float22half2_rn(make_float2(x[0], x[1]));
    }
}

// gate_apply on each of a lane's samples (two per packed fma when SPL = 2: the same IEEE
// fma per element).
template <int SPL>
__device__ __forceinline__ void gate_eval(const float4& k, const float (&a)[SPL], const float (&b)[SPL],
                                          float (&z)[SPL]) {
    if constexpr (SPL == 2) {
        const float2 av = make_float2(a[0], a[1]);
        const float2 r = __ffma2_rn(__ffma2_rn(make_float2(k.w, k.w), av, make_float2(k.z, k.z)),
                                    make_float2(b[0], b[1]), __ffma2_rn(make_float2(k.y, k.y), av, make_float2(k.x, k.x)));
        z[0] = r.x;
        z[1] = r.y;
    } else {
        z[0] = gate_apply(k, a[0], b[0]);
    }
}
// acc += ga (c0 + c1 sib) on each of a lane's samples.
template <int SPL>
__device__ __forceinline__ void edge_acc(float c0, float c1, const float (&ga)[SPL], const float (&sib)[SPL],
                                         float (&acc)[SPL]) {
    if constexpr (SPL == 2) {
        const float2 d = __ffma2_rn(make_float2(c1, c1), make_float2(sib[0], sib[1]), make_float2(c0, c0));
        const float2 r = __ffma2_rn(make_float2(ga[0], ga[1]), d, make_float2(acc[0], acc[1]));
        acc[0] = r.x;
        acc[1] = r.y;
    } else {
        acc[0] = fmaf(ga[0], fmaf(c1, sib[0], c0), acc[0]);
    }
}

// Shared-memory layout (bytes from the start of the dynamic block): act rows [n_cone][32 SPL]
// of T, adj rows [n_adj_rows][32 SPL] of float (the plan's adjoint rows: inputs, the level
// ring and the seed row), then V (and for Adam m, v) of the cone inputs, [n_cone_pi][32 SPL]
// float each (n_state = 3 rows per input with Adam, 1 with GD).
struct ResLayout {
    size_t adj, vmv, total;
};
__host__ __device__ inline ResLayout res_layout(const DevPlan& p, int act_bytes, int n_state, int spl) {
    const size_t lanes = (size_t)32 * spl;
    ResLayout r;
    r.adj = ((size_t)p.full.n_act_rows * lanes * act_bytes + 15) / 16 * 16;
    r.vmv = r.adj + (size_t)p.n_adj_rows * lanes * 4;
    r.total = r.vmv + (size_t)n_state * p.n_cone_pi * lanes * 4;
    return r;
}

template <typename T, int SPL>
__global__ void __maxnreg__(SPL == 1 ? 64 : 96) resident_steps_kernel(DevPlan p, OptParams o, float* V, float* m,
                                                                       float* v, int64_t ldv, float* loss, int t0,
                                                                       const int32_t* age, int n_steps, int64_t B) {
    constexpr int RL = res_lanes<SPL>();
    extern __shared__ __align__(16) char smem[];
    __shared__ float4 gcoef[16];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int col = lane * SPL;  // this lane's first column of every row
    const int64_t b0 = (int64_t)blockIdx.x * RL + col;
    bool valid[SPL];
#pragma unroll
    for (int q = 0; q < SPL; q++) valid[q] = b0 + q < B;
    const bool adam = o.opt == 0;
    const ResLayout lay = res_layout(p, (int)sizeof(T), adam ? 3 : 1, SPL);
    // this lane's columns of the act and adj rows (rows are < 2^27: 32-bit offsets)
    T* act = reinterpret_cast<T*>(smem) + col;
    float* adj = reinterpret_cast<float*>(smem + lay.adj) + col;
    float* sV = reinterpret_cast<float*>(smem + lay.vmv);
    float* sm = sV + (size_t)p.n_cone_pi * RL;
    float* sv = sm + (size_t)p.n_cone_pi * RL;
    const int npi = p.n_cone_pi;
    if (threadIdx.x < 16) gcoef[threadIdx.x] = gate_coeffs(threadIdx.x);
    for (int i = warp; i < npi; i += nw) {
        const int64_t r = (int64_t)__ldg(&p.cone_pi_row[i]) * ldv + b0;
#pragma unroll
        for (int q = 0; q < SPL; q++) {
            const int e = i * RL + col + q;
            sV[e] = valid[q] ? V[r + q] : 0.0f;
            if (adam) {
                sm[e] = valid[q] ? m[r + q] : 0.0f;
                sv[e] = valid[q] ? v[r + q] : 0.0f;
            }
        }
    }
    int my_age[SPL];
#pragma unroll
    for (int q = 0; q < SPL; q++) my_age[q] = age != nullptr && valid[q] ? __ldg(age + b0 + q) : 0;
    __syncthreads();
#pragma unroll 1
    for (int s = 0; s < n_steps; s++) {
        float step_size[SPL], bc2s[SPL];
#pragma unroll
        for (int q = 0; q < SPL; q++) {
            step_size[q] = bc2s[q] = 1.0f;
            if (adam) adam_bias(o, t0 + s + my_age[q], step_size[q], bc2s[q]);
        }
        // forward: the inputs' embedding, then the gate levels
        for (int i = warp; i < npi; i += nw) {
            float pv[SPL];
#pragma unroll
            for (int q = 0; q < SPL; q++) pv[q] = sigmoidf_(sV[i * RL + col + q]);
            lane_st<T, SPL>(act + i * RL, pv);
        }
        __syncthreads();
        for (int l = 1; l <= p.n_clev; l++) {
            const int lo = __ldg(&p.c_level_off[l]), hi = __ldg(&p.c_level_off[l + 1]);
            // GB gates of this warp at a time: their records and inputs are all loaded before
            // the first result is stored (a gate's inputs lie on lower levels, so no result of
            // this level is among them); the last few gates of the warp's share one by one
            constexpr int GB = 4;
            int g = lo + warp;
            for (; g + (GB - 1) * nw < hi; g += GB * nw) {
                int2 rec[GB];
                float x[GB][SPL], y[GB][SPL];
#pragma unroll
                for (int j = 0; j < GB; j++) rec[j] = __ldg(&p.full.gate[g + j * nw - npi]);
#pragma unroll
                for (int j = 0; j < GB; j++) {
                    lane_ld<T, SPL>(act + (rec[j].x & 0x0FFFFFFF) * RL, x[j]);
                    lane_ld<T, SPL>(act + rec[j].y * RL, y[j]);
                }
#pragma unroll
                for (int j = 0; j < GB; j++) {
                    float z[SPL];
                    gate_eval<SPL>(gcoef[(uint32_t)rec[j].x >> 28], x[j], y[j], z);
                    lane_st<T, SPL>(act + (g + j * nw) * RL, z);
                }
            }
            for (; g < hi; g += nw) {
                const int2 rec = __ldg(&p.full.gate[g - npi]);
                float x[SPL], y[SPL], z[SPL];
                lane_ld<T, SPL>(act + (rec.x & 0x0FFFFFFF) * RL, x);
                lane_ld<T, SPL>(act + rec.y * RL, y);
                gate_eval<SPL>(gcoef[(uint32_t)rec.x >> 28], x, y, z);
                lane_st<T, SPL>(act + g * RL, z);
            }
            __syncthreads();
        }
        // loss of the last step's forward pass, in the tiled kernel's order
        if (loss != nullptr && s == n_steps - 1 && warp == 0) {
            constexpr int NP = loss_partials<T>();
            float sum[SPL];
#pragma unroll
            for (int q = 0; q < SPL; q++) sum[q] = 0.0f;
            for (int w = 0; w < NP; w++) {
                float acc[SPL];
#pragma unroll
                for (int q = 0; q < SPL; q++) acc[q] = 0.0f;
                for (int j = w; j < p.n_out; j += NP) {
                    float yj[SPL];
                    lane_ld<T, SPL>(act + __ldg(&p.full.out_row[j]) * RL, yj);
                    const float tj = p.out_target[j];
#pragma unroll
                    for (int q = 0; q < SPL; q++) acc[q] = fmaf(yj[q] - tj, yj[q] - tj, acc[q]);
                }
#pragma unroll
                for (int q = 0; q < SPL; q++) sum[q] += acc[q];
            }
#pragma unroll
            for (int q = 0; q < SPL; q++)
                if (valid[q]) loss[b0 + q] = sum[q];
        }
        // adjoint (gather form of Eq. 8): the seed row is each sample's loss weight (1)
        if (warp == 0) {
            float one[SPL];
#pragma unroll
            for (int q = 0; q < SPL; q++) one[q] = 1.0f;
            lane_st<float, SPL>(adj + p.seed_row * RL, one);
        }
        __syncthreads();
        for (int l = p.n_clev; l >= 0; l--) {
            const int lo = l == 0 ? 0 : __ldg(&p.c_level_off[l]);
            const int hi = l == 0 ? npi : __ldg(&p.c_level_off[l + 1]);
            const int row0 = l == 0 ? 0 : (int)adj_level_row(p, l, lo);
            for (int u = lo + warp; u < hi; u += nw) {
                const int e0 = __ldg(&p.fo_off[u]), e1 = __ldg(&p.fo_off[u + 1]);
                float acc[SPL];
#pragma unroll
                for (int q = 0; q < SPL; q++) acc[q] = 0.0f;
                // EB edges at a time (records and operands loaded first, then summed in CSR
                // order), the rest one by one
                constexpr int EB = 4;
                int e = e0;
                for (; e + EB <= e1; e += EB) {
                    int4 ed[EB];
                    float ga[EB][SPL], sib[EB][SPL];
#pragma unroll
                    for (int j = 0; j < EB; j++) ed[j] = __ldg(&p.full.edge[e + j]);
#pragma unroll
                    for (int j = 0; j < EB; j++) {
                        lane_ld<float, SPL>(adj + ed[j].x * RL, ga[j]);
                        lane_ld<T, SPL>(act + (ed[j].y & 0x7FFFFFFF) * RL, sib[j]);
                    }
#pragma unroll
                    for (int j = 0; j < EB; j++)
                        edge_acc<SPL>(__int_as_float(ed[j].z), __int_as_float(ed[j].w), ga[j], sib[j], acc);
                }
                for (; e < e1; e++) {
                    const int4 ed = __ldg(&p.full.edge[e]);
                    float ga[SPL], sib[SPL];
                    lane_ld<float, SPL>(adj + ed.x * RL, ga);
                    lane_ld<T, SPL>(act + (ed.y & 0x7FFFFFFF) * RL, sib);
                    edge_acc<SPL>(__int_as_float(ed.z), __int_as_float(ed.w), ga, sib, acc);
                }
                lane_st<float, SPL>(adj + (row0 + (u - lo)) * RL, acc);
            }
            __syncthreads();
        }
        // dL/dV and the update of the inputs' V, m, v (in shared memory)
        for (int i = warp; i < npi; i += nw) {
            float pe[SPL], pbar[SPL];
            lane_ld<T, SPL>(act + i * RL, pe);
            lane_ld<float, SPL>(adj + i * RL, pbar);
#pragma unroll
            for (int q = 0; q < SPL; q++) {
                if (!valid[q]) continue;
                const int e = i * RL + col + q;
                // P = sigmoid(V): with FP32 activations the embedding row holds exactly that value
                const float P = sizeof(T) == 4 ? pe[q] : sigmoidf_(sV[e]);
                input_update_p<true>(o, sV, sm, sv, nullptr, e, sV[e], P, pbar[q], adam ? sm[e] : 0.0f,
                                     adam ? sv[e] : 0.0f, step_size[q], bc2s[q]);
            }
        }
        __syncthreads();
    }
    for (int i = warp; i < npi; i += nw) {
        const int64_t r = (int64_t)__ldg(&p.cone_pi_row[i]) * ldv + b0;
#pragma unroll
        for (int q = 0; q < SPL; q++) {
            if (!valid[q]) continue;
            const int e = i * RL + col + q;
            V[r + q] = sV[e];
            if (adam) {
                m[r + q] = sm[e];
                v[r + q] = sv[e];
            }
        }
    }
}

template <typename T, int SPL>
cudaError_t resident_launch(const DevPlan& p, const OptParams& o, float* V, float* m, float* v, int64_t ldv,
                            float* loss, int t0, const int32_t* age, int n_steps, int64_t B, int warps, size_t smem,
                            cudaStream_t s) {
    // the opt-in to the dynamic shared memory, once per type and device
    static PerDeviceOnce once;
    const cudaError_t prepared = once.run([] {
        return cudaFuncSetAttribute(resident_steps_kernel<T, SPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)RESIDENT_SMEM_MAX);
    });
    if (prepared != cudaSuccess) return prepared;
    const unsigned grid = (unsigned)((B + res_lanes<SPL>() - 1) / res_lanes<SPL>());
    resident_steps_kernel<T, SPL><<<grid, warps * 32, smem, s>>>(p, o, V, m, v, ldv, loss, t0, age, n_steps, B);
    return cudaGetLastError();
}

template <int SPL>
cudaError_t resident_dispatch(const DevPlan& p, int act_type, const OptParams& o, float* V, float* m, float* v,
                              int64_t ldv, float* loss, int t0, int n_steps, int64_t B, cudaStream_t s,
                              const int32_t* age, int warps) {
    const size_t smem = res_layout(p, act_type == ACT_F32 ? 4 : 2, o.opt == 0 ? 3 : 1, SPL).total;
    switch (act_type) {
    case ACT_F32: return resident_launch<float, SPL>(p, o, V, m, v, ldv, loss, t0, age, n_steps, B, warps, smem, s);
    case ACT_BF16:
        return resident_launch<__nv_bfloat16, SPL>(p, o, V, m, v, ldv, loss, t0, age, n_steps, B, warps, smem, s);
    default: return resident_launch<__half, SPL>(p, o, V, m, v, ldv, loss, t0, age, n_steps, B, warps, smem, s);
    }
}

}  // namespace

bool resident_config(const DevPlan& p, int act_type, int* warps, size_t* smem) {
    const ResLayout lay = res_layout(p, act_type == ACT_F32 ? 4 : 2, 3, 1);  // Adam's size: fits either way
    int widest = p.n_cone_pi;
    if (p.h_c_level_off)
        for (int l = 1; l <= p.n_clev; l++) widest = std::max(widest, p.h_c_level_off[l + 1] - p.h_c_level_off[l]);
    // two warps for narrow circuits, else one warp per 8 nodes of the widest level, up to
    // RES_MAX_WARPS (1,024 threads at 64 registers fill the register file)
    const int w = widest <= 24 ? 2 : std::min(RES_MAX_WARPS, std::max(1, (widest + 7) / 8));
    if (warps) *warps = w;
    if (smem) *smem = lay.total;
    return lay.total <= RESIDENT_SMEM_MAX && p.n_cone < (1 << 27) && p.seed_row >= 0 && p.seed_row < p.n_adj_rows;
}

bool steps_use_resident(const DevPlan& p, int act_type) {
    return p.step_kernel != STEP_KERNEL_TILED && resident_config(p, act_type, nullptr, nullptr);
}

cudaError_t launch_steps_resident(const DevPlan& p, int act_type, const OptParams& o, float* V, float* m, float* v,
                                  int64_t ldv, float* loss, int t0, int n_steps, int64_t B, cudaStream_t s,
                                  const int32_t* age) {
    if (B == 0 || n_steps <= 0) return cudaSuccess;
    int warps = 1;
    if (!resident_config(p, act_type, &warps, nullptr)) return cudaErrorInvalidValue;
    // Two samples per lane (64 per CTA) for narrow circuits on batches large enough to fill
    // the GPU many times over with half as many CTAs, when the doubled state still fits;
    // one sample per lane otherwise (small batches keep more CTAs in flight).
    constexpr int64_t SPL2_MIN_BATCH = 148 * 64 * 8;
    const bool two = warps <= 2 && B >= SPL2_MIN_BATCH &&
                     res_layout(p, act_type == ACT_F32 ? 4 : 2, 3, 2).total <= RESIDENT_SMEM_MAX;
    // Four warps then: the doubled shared memory per CTA halves the CTAs an SM holds, and
    // four warps per CTA bring back the warps per SM (measured on the paper's setting, 1M
    // samples: 0.732 ms with two warps, 0.536 with four, 0.614 with six, 0.716 with eight).
    return two ? resident_dispatch<2>(p, act_type, o, V, m, v, ldv, loss, t0, n_steps, B, s, age, 4)
               : resident_dispatch<1>(p, act_type, o, V, m, v, ldv, loss, t0, n_steps, B, s, age, warps);
}

}  // namespace sat
