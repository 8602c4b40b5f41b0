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

#include "device.hpp"
#include "relax.cuh"

namespace sat {
namespace {

constexpr int RES_LANES = 32;     // samples per CTA (one per lane)
constexpr int RES_MAX_WARPS = 32;  // warps per CTA for the widest levels

template <typename T>
struct Scalar;
template <>
struct Scalar<float> {
    static __device__ __forceinline__ float ld(const float* p) { return *p; }
    static __device__ __forceinline__ void st(float* p, float x) { *p = x; }
};
template <>
struct Scalar<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float x) { *p = __float2bfloat16_rn(x); }
};
template <>
struct Scalar<__half> {
    static __device__ __forceinline__ float ld(const __half* p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half* p, float x) { *p = __float2half_rn(x); }
};

// Shared-memory layout (bytes from the start of the dynamic block): act rows [n_cone][32]
// of T, adj rows [n_adj_rows][32] of float (the plan's adjoint rows: inputs, the level
// ring and the seed row), then V (and for Adam m, v) of the cone inputs, [n_cone_pi][32]
// float each (n_state = 3 rows per input with Adam, 1 with GD).
struct ResLayout {
    size_t adj, vmv, total;
};
__host__ __device__ inline ResLayout res_layout(const DevPlan& p, int act_bytes, int n_state) {
    ResLayout r;
    r.adj = ((size_t)p.full.n_act_rows * RES_LANES * act_bytes + 15) / 16 * 16;
    r.vmv = r.adj + (size_t)p.n_adj_rows * RES_LANES * 4;
    r.total = r.vmv + (size_t)n_state * p.n_cone_pi * RES_LANES * 4;
    return r;
}

template <typename T>
__global__ void __maxnreg__(64) resident_steps_kernel(DevPlan p, OptParams o, float* V, float* m,
                                                                           float* v, int64_t ldv, float* loss, int t0,
                                                                           const int32_t* age, int n_steps, int64_t B) {
    extern __shared__ __align__(16) char smem[];
    __shared__ float4 gcoef[16];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t b = (int64_t)blockIdx.x * RES_LANES + lane;
    const bool valid = b < B;
    const bool adam = o.opt == 0;
    const ResLayout lay = res_layout(p, (int)sizeof(T), adam ? 3 : 1);
    // this lane's column of the act and adj rows (rows are < 2^27: 32-bit offsets)
    T* act = reinterpret_cast<T*>(smem) + lane;
    float* adj = reinterpret_cast<float*>(smem + lay.adj) + lane;
    float* sV = reinterpret_cast<float*>(smem + lay.vmv);
    float* sm = sV + (size_t)p.n_cone_pi * RES_LANES;
    float* sv = sm + (size_t)p.n_cone_pi * RES_LANES;
    const int npi = p.n_cone_pi;
    if (threadIdx.x < 16) gcoef[threadIdx.x] = gate_coeffs(threadIdx.x);
    for (int i = warp; i < npi; i += nw) {
        const int64_t r = (int64_t)__ldg(&p.cone_pi_row[i]) * ldv + b;
        const int e = i * RES_LANES + lane;
        sV[e] = valid ? V[r] : 0.0f;
        if (adam) {
            sm[e] = valid ? m[r] : 0.0f;
            sv[e] = valid ? v[r] : 0.0f;
        }
    }
    const int my_age = age != nullptr && valid ? __ldg(age + b) : 0;
    __syncthreads();
#pragma unroll 1
    for (int s = 0; s < n_steps; s++) {
        float step_size = 1.0f, bc2s = 1.0f;
        if (adam) adam_bias(o, t0 + s + my_age, step_size, bc2s);
        // forward: the inputs' embedding, then the gate levels
        for (int i = warp; i < npi; i += nw) Scalar<T>::st(act + i * RES_LANES, sigmoidf_(sV[i * RES_LANES + lane]));
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
                float x[GB], y[GB];
#pragma unroll
                for (int j = 0; j < GB; j++) rec[j] = __ldg(&p.full.gate[g + j * nw - npi]);
#pragma unroll
                for (int j = 0; j < GB; j++) {
                    x[j] = Scalar<T>::ld(act + (rec[j].x & 0x0FFFFFFF) * RES_LANES);
                    y[j] = Scalar<T>::ld(act + rec[j].y * RES_LANES);
                }
#pragma unroll
                for (int j = 0; j < GB; j++)
                    Scalar<T>::st(act + (g + j * nw) * RES_LANES, gate_apply(gcoef[(uint32_t)rec[j].x >> 28], x[j], y[j]));
            }
            for (; g < hi; g += nw) {
                const int2 rec = __ldg(&p.full.gate[g - npi]);
                const float x = Scalar<T>::ld(act + (rec.x & 0x0FFFFFFF) * RES_LANES);
                const float y = Scalar<T>::ld(act + rec.y * RES_LANES);
                Scalar<T>::st(act + g * RES_LANES, gate_apply(gcoef[(uint32_t)rec.x >> 28], x, y));
            }
            __syncthreads();
        }
        // loss of the last step's forward pass, in the tiled kernel's order
        if (loss != nullptr && s == n_steps - 1 && warp == 0) {
            constexpr int NP = loss_partials<T>();
            float sum = 0.0f;
            for (int w = 0; w < NP; w++) {
                float acc = 0.0f;
                for (int j = w; j < p.n_out; j += NP) {
                    const float yj = Scalar<T>::ld(act + __ldg(&p.full.out_row[j]) * RES_LANES);
                    const float tj = p.out_target[j];
                    acc = fmaf(yj - tj, yj - tj, acc);
                }
                sum += acc;
            }
            if (valid) loss[b] = sum;
        }
        // adjoint (gather form of Eq. 8): the seed row is each sample's loss weight (1)
        if (warp == 0) adj[p.seed_row * RES_LANES] = 1.0f;
        __syncthreads();
        for (int l = p.n_clev; l >= 0; l--) {
            const int lo = l == 0 ? 0 : __ldg(&p.c_level_off[l]);
            const int hi = l == 0 ? npi : __ldg(&p.c_level_off[l + 1]);
            const int row0 = l == 0 ? 0 : (int)adj_level_row(p, l, lo);
            for (int u = lo + warp; u < hi; u += nw) {
                const int e0 = __ldg(&p.fo_off[u]), e1 = __ldg(&p.fo_off[u + 1]);
                float acc = 0.0f;
                // EB edges at a time (records and operands loaded first, then summed in CSR
                // order), the rest one by one
                constexpr int EB = 4;
                int e = e0;
                for (; e + EB <= e1; e += EB) {
                    int4 ed[EB];
                    float ga[EB], sib[EB];
#pragma unroll
                    for (int j = 0; j < EB; j++) ed[j] = __ldg(&p.full.edge[e + j]);
#pragma unroll
                    for (int j = 0; j < EB; j++) {
                        ga[j] = adj[ed[j].x * RES_LANES];
                        sib[j] = Scalar<T>::ld(act + (ed[j].y & 0x7FFFFFFF) * RES_LANES);
                    }
#pragma unroll
                    for (int j = 0; j < EB; j++)
                        acc = fmaf(ga[j], fmaf(__int_as_float(ed[j].w), sib[j], __int_as_float(ed[j].z)), acc);
                }
                for (; e < e1; e++) {
                    const int4 ed = __ldg(&p.full.edge[e]);
                    const float ga = adj[ed.x * RES_LANES];
                    const float sib = Scalar<T>::ld(act + (ed.y & 0x7FFFFFFF) * RES_LANES);
                    acc = fmaf(ga, fmaf(__int_as_float(ed.w), sib, __int_as_float(ed.z)), acc);
                }
                adj[(row0 + (u - lo)) * RES_LANES] = acc;
            }
            __syncthreads();
        }
        // dL/dV and the update of the inputs' V, m, v (in shared memory)
        if (valid)
            for (int i = warp; i < npi; i += nw) {
                const int e = i * RES_LANES + lane;
                // P = sigmoid(V): with FP32 activations the embedding row holds exactly that value
                const float P = sizeof(T) == 4 ? Scalar<T>::ld(act + i * RES_LANES) : sigmoidf_(sV[e]);
                input_update_p<true>(o, sV, sm, sv, nullptr, e, sV[e], P, adj[i * RES_LANES], adam ? sm[e] : 0.0f,
                                     adam ? sv[e] : 0.0f, step_size, bc2s);
            }
        __syncthreads();
    }
    if (valid)
        for (int i = warp; i < npi; i += nw) {
            const int64_t r = (int64_t)__ldg(&p.cone_pi_row[i]) * ldv + b;
            const int e = i * RES_LANES + lane;
            V[r] = sV[e];
            if (adam) {
                m[r] = sm[e];
                v[r] = sv[e];
            }
        }
}

template <typename T>
cudaError_t resident_launch(const DevPlan& p, const OptParams& o, float* V, float* m, float* v, int64_t ldv,
                            float* loss, int t0, const int32_t* age, int n_steps, int64_t B, int warps, size_t smem,
                            cudaStream_t s) {
    // the opt-in to the dynamic shared memory, once per type and device
    static PerDeviceOnce once;
    const cudaError_t prepared = once.run([] {
        return cudaFuncSetAttribute(resident_steps_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)RESIDENT_SMEM_MAX);
    });
    if (prepared != cudaSuccess) return prepared;
    const unsigned grid = (unsigned)((B + RES_LANES - 1) / RES_LANES);
    resident_steps_kernel<T><<<grid, warps * 32, smem, s>>>(p, o, V, m, v, ldv, loss, t0, age, n_steps, B);
    return cudaGetLastError();
}

}  // namespace

bool resident_config(const DevPlan& p, int act_type, int* warps, size_t* smem) {
    const ResLayout lay = res_layout(p, act_type == ACT_F32 ? 4 : 2, 3);  // Adam's size: fits either way
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
    const size_t smem = res_layout(p, act_type == ACT_F32 ? 4 : 2, o.opt == 0 ? 3 : 1).total;
    switch (act_type) {
    case ACT_F32: return resident_launch<float>(p, o, V, m, v, ldv, loss, t0, age, n_steps, B, warps, smem, s);
    case ACT_BF16:
        return resident_launch<__nv_bfloat16>(p, o, V, m, v, ldv, loss, t0, age, n_steps, B, warps, smem, s);
    default: return resident_launch<__half>(p, o, V, m, v, ldv, loss, t0, age, n_steps, B, warps, smem, s);
    }
}

}  // namespace sat
