// CUDA kernels of the sampler's hot path (sm_103a).
//
// Layout: every per-sample quantity is stored node-major with the batch
// contiguous ("SoA"): row r of V, m, v, gV is primary input r over the batch;
// row u of act / adj is cone node u over the batch.  A CTA owns a tile of 32
// samples (lane = sample) and walks the levels of the circuit; samples are
// independent, so the only synchronisation is __syncthreads between levels.
//
// Relaxation (Table 1): AND a*b, OR 1-(1-a)(1-b), XOR a+b-2ab, input negation
// 1-a; embedding P = sigmoid(V) (Eq. 5); loss sum_j (Y_j - T_j)^2 (Eq. 7); the
// adjoint is the chain rule of Eq. 8 in gather form (each node sums, in a fixed
// order, the contributions of its fan-out edges); the update is Eq. 9 (GD) or
// Adam in PyTorch's formulation.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "device.hpp"

namespace sat {
namespace {

constexpr int VEC = 2;                 // consecutive samples per lane
constexpr int TILE = 32 * VEC;         // samples per CTA
constexpr int STEP_THREADS = 512;
constexpr int UBATCH = 2;              // input rows per warp in the input-level passes
constexpr unsigned FULL = 0xffffffffu;

// Two consecutive samples of one scratch row, in registers as float2.
template <typename T> struct ActIO;
template <> struct ActIO<float> {
    static __device__ __forceinline__ float2 ld(const float* p) { return *reinterpret_cast<const float2*>(p); }
    static __device__ __forceinline__ void st(float* p, float2 x) { *reinterpret_cast<float2*>(p) = x; }
};
template <> struct ActIO<__nv_bfloat16> {
    static __device__ __forceinline__ float2 ld(const __nv_bfloat16* p) {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float2 x) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __float22bfloat162_rn(x);
    }
};
template <> struct ActIO<__half> {
    static __device__ __forceinline__ float2 ld(const __half* p) {
        return __half22float2(*reinterpret_cast<const __half2*>(p));
    }
    static __device__ __forceinline__ void st(__half* p, float2 x) { *reinterpret_cast<__half2*>(p) = __float22half2_rn(x); }
};

__device__ __forceinline__ float sigmoidf_(float v) { return 1.0f / (1.0f + expf(-v)); }

// Table 1 on (possibly negated) inputs; gop = op | neg0 << 2 | neg1 << 3.
__device__ __forceinline__ float gate_eval(uint32_t gop, float a, float b) {
    if (gop & 4) a = 1.0f - a;
    if (gop & 8) b = 1.0f - b;
    switch (gop & 3) {
    case 0: return a * b;
    case 1: return fmaf(-a, b, a + b);
    default: return fmaf(-2.0f * a, b, a + b);
    }
}

__device__ __forceinline__ float2 gate_eval2(uint32_t gop, float2 a, float2 b) {
    return make_float2(gate_eval(gop, a.x, b.x), gate_eval(gop, a.y, b.y));
}

struct TileCtx {
    int lane, warp, nw;
    int64_t b;      // first of this lane's VEC samples
    bool ok0, ok1;  // b < B, b + 1 < B
};

__device__ __forceinline__ TileCtx tile_ctx(int64_t B) {
    TileCtx c;
    c.lane = threadIdx.x & 31;
    c.warp = threadIdx.x >> 5;
    c.nw = blockDim.x >> 5;
    c.b = (int64_t)blockIdx.x * TILE + c.lane * VEC;
    c.ok0 = c.b < B;
    c.ok1 = c.b + 1 < B;
    return c;
}

// Element offset of this lane's samples in row `row` of a tile's [n_cone][TILE] block.
__device__ __forceinline__ uint32_t at(int row, const TileCtx& c) {
    return (uint32_t)row * TILE + (uint32_t)(c.lane * VEC);
}

// Adam bias corrections (PyTorch: step_size = lr / (1 - b1^t), sqrt(1 - b2^t)),
// from the running powers b1^t, b2^t kept in double like its host scalars.
__device__ __forceinline__ void adam_bias(const OptParams& o, double p1, double p2, float& step_size, float& bc2s) {
    step_size = (float)((double)o.lr / (1.0 - p1));
    bc2s = (float)sqrt(1.0 - p2);
}

// ------------------------------------------------------ async row copies --
// Rows of a tile's scratch block are staged into shared memory by the bulk
// copy engine (cp.async.bulk, one instruction per row, completion counted in
// bytes on an mbarrier).  Each warp owns NSLOT slots and keeps NSLOT-1 chunks
// in flight while it computes on the oldest one.  Every mbarrier wait is
// bounded: on expiry the kernel records STATUS_WAIT_TIMEOUT in the plan's
// status word and carries on (results are then invalid, the GPU is not hung).
constexpr int CHUNK = 8;   // gates (forward) or fan-out edges (adjoint) per chunk
constexpr int NSLOT = 3;   // pipeline depth per warp
constexpr unsigned STATUS_WAIT_TIMEOUT = 4u;
constexpr uint32_t WAIT_LIMIT = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Global -> shared bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Per-warp staging state: NSLOT slots of slot_bytes<T>() and their mbarriers.
struct Stage {
    char* buf;
    uint64_t* bar;
    uint32_t parity;      // bit s: parity of the next completion of slot s
    unsigned* status;     // plan status word (device)
    bool poisoned;        // a wait expired: stop waiting, results are invalid
};

// Bytes of one slot: the 2 CHUNK input rows of CHUNK gates (forward) or CHUNK
// fp32 adjoint rows plus CHUNK act rows (adjoint).
template <typename T>
__host__ __device__ constexpr int slot_bytes() {
    return (2 * CHUNK * TILE * (int)sizeof(T)) > (CHUNK * TILE * 4 + CHUNK * TILE * (int)sizeof(T))
               ? (2 * CHUNK * TILE * (int)sizeof(T))
               : (CHUNK * TILE * 4 + CHUNK * TILE * (int)sizeof(T));
}
// Per-warp stride, rounded to 128 bytes so every slot (and every bulk-copy
// destination inside it) stays 16-byte aligned for every warp.
template <typename T>
__host__ __device__ constexpr int warp_stage_bytes() {
    return (NSLOT * slot_bytes<T>() + NSLOT * 8 + 127) / 128 * 128;
}

template <typename T>
__device__ __forceinline__ Stage make_stage(char* smem, unsigned* status, const TileCtx& c) {
    Stage st;
    st.buf = smem + c.warp * warp_stage_bytes<T>();
    st.bar = reinterpret_cast<uint64_t*>(st.buf + NSLOT * slot_bytes<T>());
    st.parity = 0;
    st.status = status;
    st.poisoned = false;
    return st;
}

// Warp-uniform: wait for the completion of slot s.
__device__ __forceinline__ void stage_wait(Stage& st, int s) {
    if (!st.poisoned) {
        uint32_t it = 0;
        while (!mbar_try_wait(st.bar + s, (st.parity >> s) & 1u)) {
            if (++it >= WAIT_LIMIT) {
                st.poisoned = true;
                if ((threadIdx.x & 31) == 0) atomicOr(st.status, STATUS_WAIT_TIMEOUT);
                break;
            }
        }
    }
    st.parity ^= 1u << s;
    __syncwarp();
}

// Forward pass of one tile: P = sigmoid(V) for the cone inputs, then every cone
// level.  Within a level each warp takes a contiguous run of gates; 32 gate
// records come in one coalesced load and are broadcast by shuffles; the two
// input rows of each gate are bulk-copied into shared memory, CHUNK gates per
// slot, NSLOT-1 chunks ahead of the computation.
template <typename T>
__device__ void tile_forward(const DevPlan& p, const float* __restrict__ V, int64_t ldv, T* act, Stage& st,
                             const TileCtx& c) {
    constexpr int ROWB = TILE * (int)sizeof(T);
    constexpr int SLOT = slot_bytes<T>();
    for (int i0 = c.warp * UBATCH; i0 < p.n_cone_pi; i0 += c.nw * UBATCH) {
        float2 x[UBATCH];
#pragma unroll
        for (int u = 0; u < UBATCH; u++) {
            const int i = i0 + u;
            x[u] = make_float2(0.0f, 0.0f);
            if (i < p.n_cone_pi) {
                const float* r = V + (int64_t)__ldg(&p.cone_pi_row[i]) * ldv + c.b;
                if (c.ok0) x[u].x = r[0];
                if (c.ok1) x[u].y = r[1];
            }
        }
#pragma unroll
        for (int u = 0; u < UBATCH; u++) {
            const int i = i0 + u;
            if (i < p.n_cone_pi) ActIO<T>::st(act + at(i, c), make_float2(sigmoidf_(x[u].x), sigmoidf_(x[u].y)));
        }
    }
    fence_async_global();
    __syncthreads();
    const char* abytes = reinterpret_cast<const char*>(act);
    for (int l = 1; l <= p.n_clev; l++) {
        const int lo = __ldg(&p.c_level_off[l]), hi = __ldg(&p.c_level_off[l + 1]);
        const int per = (hi - lo + c.nw - 1) / c.nw;
        const int g0 = lo + c.warp * per, g1 = min(g0 + per, hi);
        for (int base = g0; base < g1; base += 32) {
            const int cnt = min(32, g1 - base);
            int2 mine = make_int2(0, 0);
            if (c.lane < cnt) mine = __ldg(&p.c_gate[base + c.lane - p.n_cone_pi]);
            const int nch = (cnt + CHUNK - 1) / CHUNK;
            auto issue = [&](int ch) {
                const int s = ch % NSLOT;
                const int ne = min(CHUNK, cnt - ch * CHUNK);
                const int src = ch * CHUNK + (c.lane >> 1);
                const int x = __shfl_sync(FULL, mine.x, src & 31) & 0x0FFFFFFF;
                const int y = __shfl_sync(FULL, mine.y, src & 31);
                if (c.lane == 0) mbar_expect_tx(st.bar + s, (uint32_t)(2 * ne * ROWB));
                __syncwarp();
                if (c.lane < 2 * ne)
                    bulk_g2s(st.buf + s * SLOT + c.lane * ROWB, abytes + (size_t)((c.lane & 1) ? y : x) * ROWB, ROWB,
                             st.bar + s);
            };
            for (int ch = 0; ch < NSLOT - 1 && ch < nch; ch++) issue(ch);
            for (int ch = 0; ch < nch; ch++) {
                if (ch + NSLOT - 1 < nch) issue(ch + NSLOT - 1);
                const int s = ch % NSLOT;
                stage_wait(st, s);
                const char* sb = st.buf + s * SLOT;
#pragma unroll
                for (int j = 0; j < CHUNK; j++) {
                    const int gl = ch * CHUNK + j;
                    const uint32_t gop = (uint32_t)__shfl_sync(FULL, mine.x, gl & 31) >> 28;
                    if (gl < cnt) {
                        const float2 x = ActIO<T>::ld(reinterpret_cast<const T*>(sb + (2 * j) * ROWB) + c.lane * VEC);
                        const float2 y = ActIO<T>::ld(reinterpret_cast<const T*>(sb + (2 * j + 1) * ROWB) + c.lane * VEC);
                        ActIO<T>::st(act + at(base + gl, c), gate_eval2(gop, x, y));
                    }
                }
                fence_async_shared();
                __syncwarp();
            }
        }
        fence_async_global();
        __syncthreads();
    }
}

// Per-sample loss sum_j (Y_j - T_j)^2, FP32, fixed order (warp-strided partials, then warp order).
template <typename T>
__device__ void tile_loss(const DevPlan& p, const T* act, float* loss, const TileCtx& c) {
    __shared__ float2 part[STEP_THREADS / 32][32];
    float2 acc = make_float2(0.0f, 0.0f);
    for (int j = c.warp; j < p.n_out; j += c.nw) {
        const float2 y = ActIO<T>::ld(act + at(p.c_out_node[j], c));
        const float t = p.out_target[j];
        acc.x = fmaf(y.x - t, y.x - t, acc.x);
        acc.y = fmaf(y.y - t, y.y - t, acc.y);
    }
    part[c.warp][c.lane] = acc;
    __syncthreads();
    if (c.warp == 0) {
        float2 s = make_float2(0.0f, 0.0f);
        for (int w = 0; w < c.nw; w++) {
            s.x += part[w][c.lane].x;
            s.y += part[w][c.lane].y;
        }
        if (c.ok0) loss[c.b] = s.x;
        if (c.ok1) loss[c.b + 1] = s.y;
    }
    __syncthreads();
}

// Adjoints of cone nodes [lo, hi) (gather form of Eq. 8): each warp takes a
// contiguous run of nodes, whose fan-out edges are contiguous in the CSR and
// are summed in CSR order.  An edge contributes ga * (c0 + c1 * A_sibling)
// with ga the consumer's adjoint, or seed_scale for an output seed.  The
// consumer-adjoint and sibling rows are bulk-copied into shared memory, CHUNK
// edges per slot.
template <typename T>
__device__ void level_adjoint(const DevPlan& p, int lo, int hi, const T* act, float* adj, float2 seed_scale,
                              Stage& st, const TileCtx& c) {
    constexpr int ROWB = TILE * (int)sizeof(T);
    constexpr int ROWF = TILE * 4;
    constexpr int SLOT = slot_bytes<T>();
    const char* abytes = reinterpret_cast<const char*>(act);
    const char* gbytes = reinterpret_cast<const char*>(adj);
    const int per = (hi - lo + c.nw - 1) / c.nw;
    const int u0 = lo + c.warp * per, u1 = min(u0 + per, hi);
    for (int ua = u0; ua < u1; ua += 31) {
        const int nn = min(31, u1 - ua);
        const int off = (c.lane <= nn) ? __ldg(&p.fo_off[ua + c.lane]) : 0;
        const int e_begin = __shfl_sync(FULL, off, 0), e_end = __shfl_sync(FULL, off, nn);
        int k = 0;
        int k_end = __shfl_sync(FULL, off, 1);
        float2 acc = make_float2(0.0f, 0.0f);
        for (int base = e_begin; base < e_end; base += 32) {
            const int cnt = min(32, e_end - base);
            int4 mine = make_int4(-1, 0, 0, 0);
            if (c.lane < cnt) mine = __ldg(&p.fo_edge[base + c.lane]);
            const int nch = (cnt + CHUNK - 1) / CHUNK;
            auto issue = [&](int ch) {
                const int s = ch % NSLOT;
                const int ne = min(CHUNK, cnt - ch * CHUNK);
                const int j = c.lane & (CHUNK - 1);
                const int src = (ch * CHUNK + j) & 31;
                const int g = __shfl_sync(FULL, mine.x, src);
                const int sib = __shfl_sync(FULL, mine.y, src);
                const bool adj_row = c.lane < CHUNK && j < ne && g >= 0;
                const bool act_row = c.lane >= CHUNK && c.lane < 2 * CHUNK && j < ne;
                const uint32_t nadj = __popc(__ballot_sync(FULL, adj_row));
                if (c.lane == 0) mbar_expect_tx(st.bar + s, nadj * ROWF + (uint32_t)ne * ROWB);
                __syncwarp();
                char* sb = st.buf + s * SLOT;
                if (adj_row) bulk_g2s(sb + j * ROWF, gbytes + (size_t)g * ROWF, ROWF, st.bar + s);
                if (act_row) bulk_g2s(sb + CHUNK * ROWF + j * ROWB, abytes + (size_t)sib * ROWB, ROWB, st.bar + s);
            };
            for (int ch = 0; ch < NSLOT - 1 && ch < nch; ch++) issue(ch);
            for (int ch = 0; ch < nch; ch++) {
                if (ch + NSLOT - 1 < nch) issue(ch + NSLOT - 1);
                const int s = ch % NSLOT;
                stage_wait(st, s);
                const char* sb = st.buf + s * SLOT;
#pragma unroll
                for (int j = 0; j < CHUNK; j++) {
                    const int el = ch * CHUNK + j;
                    const int gx = __shfl_sync(FULL, mine.x, el & 31);
                    const float c0 = (float)__shfl_sync(FULL, mine.z, el & 31);
                    const float c1 = (float)__shfl_sync(FULL, mine.w, el & 31);
                    if (el < cnt) {
                        const int e = base + el;
                        while (e >= k_end) {
                            *reinterpret_cast<float2*>(adj + at(ua + k, c)) = acc;
                            acc = make_float2(0.0f, 0.0f);
                            k++;
                            k_end = __shfl_sync(FULL, off, k + 1);
                        }
                        const float2 ga = gx < 0 ? seed_scale
                                                 : *reinterpret_cast<const float2*>(sb + j * ROWF + c.lane * 8);
                        const float2 sv =
                            ActIO<T>::ld(reinterpret_cast<const T*>(sb + CHUNK * ROWF + j * ROWB) + c.lane * VEC);
                        acc.x = fmaf(ga.x, fmaf(c1, sv.x, c0), acc.x);
                        acc.y = fmaf(ga.y, fmaf(c1, sv.y, c0), acc.y);
                    }
                }
                fence_async_shared();
                __syncwarp();
            }
        }
        while (k < nn) {
            *reinterpret_cast<float2*>(adj + at(ua + k, c)) = acc;
            acc = make_float2(0.0f, 0.0f);
            k++;
        }
    }
}

// dL/dV = Pbar * P (1 - P) for one sample, then GD (Eq. 9) or Adam (PyTorch's
// formulation, no weight decay) on V, m, v at element r.
template <bool UPDATE>
__device__ __forceinline__ void input_update(const OptParams& o, float* V, float* m, float* v, float* gV, int64_t r,
                                             float vv, float pbar, float mm, float ss, float step_size, float bc2s) {
    const float P = sigmoidf_(vv);
    const float g = pbar * P * (1.0f - P);
    if (!UPDATE) {
        gV[r] = g;
    } else if (o.opt == 1) {
        V[r] = fmaf(-o.lr, g, vv);
    } else {
        const float m1 = fmaf(1.0f - o.b1, g - mm, mm);
        const float v1 = fmaf(o.b2, ss, (1.0f - o.b2) * g * g);
        m[r] = m1;
        v[r] = v1;
        V[r] = vv - step_size * (m1 / (sqrtf(v1) / bc2s + o.eps));
    }
}

// Backward pass of one tile over levels n_clev..0.  The input level's adjoints
// (of P) are turned into dL/dV and either stored (gV) or applied by the
// optimiser, UBATCH rows at a time.
template <typename T, bool UPDATE>
__device__ void tile_backward(const DevPlan& p, const OptParams& o, float* V, float* m, float* v, float* gV,
                              int64_t ldv, const T* act, float* adj, const float* grad_loss, double p1, double p2,
                              Stage& st, const TileCtx& c) {
    float2 seed_scale = make_float2(1.0f, 1.0f);
    if (grad_loss != nullptr) {
        seed_scale.x = c.ok0 ? grad_loss[c.b] : 0.0f;
        seed_scale.y = c.ok1 ? grad_loss[c.b + 1] : 0.0f;
    }
    for (int l = p.n_clev; l >= 0; l--) {
        const int lo = l == 0 ? 0 : __ldg(&p.c_level_off[l]);
        const int hi = l == 0 ? p.n_cone_pi : __ldg(&p.c_level_off[l + 1]);
        level_adjoint<T>(p, lo, hi, act, adj, seed_scale, st, c);
        fence_async_global();
        __syncthreads();
    }
    float step_size = 0.0f, bc2s = 1.0f;
    if (UPDATE && o.opt == 0) adam_bias(o, p1, p2, step_size, bc2s);
    const bool adam = UPDATE && o.opt == 0;
    for (int i0 = c.warp * UBATCH; i0 < p.n_cone_pi; i0 += c.nw * UBATCH) {
        float2 vv[UBATCH], pb[UBATCH], mm[UBATCH], ss[UBATCH];
        int64_t r[UBATCH];
#pragma unroll
        for (int u = 0; u < UBATCH; u++) {
            const int i = i0 + u;
            if (i < p.n_cone_pi) {
                r[u] = (int64_t)__ldg(&p.cone_pi_row[i]) * ldv + c.b;
                pb[u] = *reinterpret_cast<const float2*>(adj + at(i, c));
                vv[u] = mm[u] = ss[u] = make_float2(0.0f, 0.0f);
                if (c.ok0) {
                    vv[u].x = V[r[u]];
                    if (adam) { mm[u].x = m[r[u]]; ss[u].x = v[r[u]]; }
                }
                if (c.ok1) {
                    vv[u].y = V[r[u] + 1];
                    if (adam) { mm[u].y = m[r[u] + 1]; ss[u].y = v[r[u] + 1]; }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < UBATCH; u++) {
            if (i0 + u >= p.n_cone_pi) continue;
            if (c.ok0) input_update<UPDATE>(o, V, m, v, gV, r[u], vv[u].x, pb[u].x, mm[u].x, ss[u].x, step_size, bc2s);
            if (c.ok1) input_update<UPDATE>(o, V, m, v, gV, r[u] + 1, vv[u].y, pb[u].y, mm[u].y, ss[u].y, step_size, bc2s);
        }
    }
    __syncthreads();
}

// Scratch of tile t: act / adj rows [n_cone][TILE] starting at element t * n_cone * TILE.
// Dynamic shared memory: warp_stage_bytes<T>() per warp (slots + mbarriers).
template <typename T>
__device__ __forceinline__ Stage init_stage(char* smem, const DevPlan& p, const TileCtx& c) {
    Stage st = make_stage<T>(smem, p.status, c);
    if (c.lane == 0)
        for (int s = 0; s < NSLOT; s++) mbar_init(st.bar + s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();
    return st;
}

template <typename T>
__global__ void __launch_bounds__(STEP_THREADS, 1) forward_kernel(DevPlan p, const float* V, int64_t ldv, T* act,
                                                                  float* loss, int64_t B) {
    extern __shared__ __align__(128) char smem[];
    const TileCtx c = tile_ctx(B);
    Stage st = init_stage<T>(smem, p, c);
    T* a = act + (size_t)blockIdx.x * (size_t)p.n_cone * TILE;
    tile_forward<T>(p, V, ldv, a, st, c);
    if (loss) tile_loss<T>(p, a, loss, c);
}

template <typename T>
__global__ void __launch_bounds__(STEP_THREADS, 1) backward_kernel(DevPlan p, const float* V, int64_t ldv,
                                                                   const T* act, float* adj, const float* grad_loss,
                                                                   float* gV, int64_t B) {
    extern __shared__ __align__(128) char smem[];
    const TileCtx c = tile_ctx(B);
    Stage st = init_stage<T>(smem, p, c);
    const size_t off = (size_t)blockIdx.x * (size_t)p.n_cone * TILE;
    OptParams o;
    tile_backward<T, false>(p, o, const_cast<float*>(V), nullptr, nullptr, gV, ldv, act + off, adj + off, grad_loss,
                            0.0, 0.0, st, c);
}

// The fused hot loop: n_steps x (forward, loss, adjoint, update) for one tile;
// p1, p2 = b1^(t0-1), b2^(t0-1).
template <typename T>
__global__ void __launch_bounds__(STEP_THREADS, 1) steps_kernel(DevPlan p, OptParams o, float* V, float* m, float* v,
                                                                int64_t ldv, T* act, float* adj, float* loss,
                                                                double p1, double p2, int n_steps, int64_t B) {
    extern __shared__ __align__(128) char smem[];
    const TileCtx c = tile_ctx(B);
    Stage st = init_stage<T>(smem, p, c);
    const size_t off = (size_t)blockIdx.x * (size_t)p.n_cone * TILE;
    T* a = act + off;
    float* g = adj + off;
#pragma unroll 1
    for (int s = 0; s < n_steps; s++) {
        p1 *= (double)o.b1;
        p2 *= (double)o.b2;
        tile_forward<T>(p, V, ldv, a, st, c);
        if (loss && s == n_steps - 1) tile_loss<T>(p, a, loss, c);
        tile_backward<T, true>(p, o, V, m, v, nullptr, ldv, a, g, nullptr, p1, p2, st, c);
    }
}

template <typename T>
constexpr size_t stage_smem() {
    return (size_t)(STEP_THREADS / 32) * warp_stage_bytes<T>();
}

// Opt the step kernels into the dynamic shared memory they use (once per type).
template <typename T>
cudaError_t prepare_tile_kernels() {
    static cudaError_t done = [] {
        const int bytes = (int)stage_smem<T>();
        cudaError_t e = cudaFuncSetAttribute(forward_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(backward_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(steps_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        return e;
    }();
    return done;
}

__global__ void opt_update_kernel(DevPlan p, OptParams o, float* V, float* m, float* v, const float* gV, int64_t ldv,
                                  double p1, double p2, int64_t B) {
    const int64_t n = (int64_t)p.n_cone_pi * B;
    float step_size = 0.0f, bc2s = 1.0f;
    adam_bias(o, p1, p2, step_size, bc2s);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k / B, b = k % B;
        const int64_t r = (int64_t)p.cone_pi_row[i] * ldv + b;
        const float g = gV[r];
        if (o.opt == 1) {
            V[r] = fmaf(-o.lr, g, V[r]);
        } else {
            float mm = m[r], vv = v[r];
            mm = fmaf(1.0f - o.b1, g - mm, mm);
            vv = fmaf(o.b2, vv, (1.0f - o.b2) * g * g);
            m[r] = mm;
            v[r] = vv;
            V[r] = V[r] - step_size * (mm / (sqrtf(vv) / bc2s + o.eps));
        }
    }
}

// ------------------------------------------------------------ init -------
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

// V[r][b] = scale * sqrt(-2 ln u1) cos(2 pi u2), (u1, u2) from counter (b, r, round, 0).
__global__ void init_normal_kernel(int32_t n_pi, uint64_t seed, uint32_t round, float scale, float* V, int64_t ldv,
                                   int64_t B) {
    const int64_t n = (int64_t)n_pi * B;
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = k / B, b = k % B;
        const uint4 o = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)r, round, 0u), key);
        const float u1 = (float)((o.x >> 8) + 1u) * (1.0f / 16777216.0f);
        const float u2 = (float)(o.y >> 8) * (1.0f / 16777216.0f);
        V[r * ldv + b] = scale * sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
    }
}

// ---------------------------------------------------- verification -------
// Threshold (bit = V > 0) of a 32 x 32 (sample x input) tile: ballots give the
// bitsliced input rows; a shared-memory transpose gives per-sample keys.
__global__ void threshold_kernel(const float* V, int64_t ldv, int32_t n_pi, uint32_t* bits, int64_t ldw,
                                 uint32_t* keys, int32_t kw, int64_t B) {
    __shared__ float tile[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t b0 = (int64_t)blockIdx.x * 32, pi0 = (int64_t)blockIdx.y * 32;
    const int64_t pi = pi0 + ty, b = b0 + tx;
    const float val = (pi < n_pi && b < B) ? V[pi * ldv + b] : 0.0f;
    tile[ty][tx] = val;
    const unsigned wb = __ballot_sync(0xffffffffu, val > 0.0f);
    if (tx == 0 && pi < n_pi) bits[pi * ldw + blockIdx.x] = wb;
    __syncthreads();
    const float u = tile[tx][ty];
    const unsigned wk = __ballot_sync(0xffffffffu, u > 0.0f);
    if (tx == 0 && b0 + ty < B) keys[(b0 + ty) * kw + blockIdx.y] = wk;
}

// Boolean pass over every gate (constrained or not), 32 samples per word.
template <int TW>
__global__ void __launch_bounds__(512) hard_eval_kernel(DevPlan p, uint32_t* bits, int64_t ldw, int64_t W) {
    constexpr int GPW = 32 / TW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int sub = lane / TW;
    const int64_t w = (int64_t)blockIdx.x * TW + lane % TW;
    const bool ok = w < W;
    for (int l = 1; l <= p.n_flev; l++) {
        const int lo = p.f_level_off[l], hi = p.f_level_off[l + 1];
        for (int g = lo + warp * GPW + sub; g < hi; g += nw * GPW) {
            if (!ok) continue;
            const int2 gm = __ldg(&p.f_gate[g - p.n_pi]);
            const uint32_t gop = (uint32_t)gm.x >> 28;
            uint32_t a = bits[(int64_t)(gm.x & 0x0FFFFFFF) * ldw + w];
            uint32_t b = bits[(int64_t)gm.y * ldw + w];
            if (gop & 4) a = ~a;
            if (gop & 8) b = ~b;
            const uint32_t op = gop & 3;
            bits[(int64_t)g * ldw + w] = op == 0 ? (a & b) : op == 1 ? (a | b) : (a ^ b);
        }
        __syncthreads();
    }
}

__global__ void valid_init_kernel(uint32_t* valid, int64_t W, int64_t B) {
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    const int rem = (int)(B - w * 32);
    valid[w] = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
}

// Every original clause must hold a true literal (Section II-A); the AND over a
// chunk of clauses is folded into valid[] with atomicAnd.
constexpr int CLAUSES_PER_CTA = 2048;
__global__ void __launch_bounds__(256) cnf_check_kernel(DevPlan p, const uint32_t* bits, int64_t ldw, uint32_t* valid,
                                                        int64_t W) {
    __shared__ uint32_t red[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t w = (int64_t)blockIdx.x * 32 + lane;
    const bool ok = w < W;
    const int64_t c0 = (int64_t)blockIdx.y * CLAUSES_PER_CTA;
    const int64_t c1 = min(c0 + CLAUSES_PER_CTA, p.n_clauses);
    uint32_t acc = 0xffffffffu;
    if (ok) {
        for (int64_t cl = c0 + warp; cl < c1; cl += nw) {
            uint32_t any = 0;
            for (int64_t i = p.cl_off[cl], e = p.cl_off[cl + 1]; i < e; i++) {
                const int32_t L = __ldg(&p.cl_lit[i]);
                const uint32_t x = bits[(int64_t)(L >> 1) * ldw + w];
                any |= (L & 1) ? ~x : x;
            }
            acc &= any;
        }
    }
    red[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && ok) {
        uint32_t r = 0xffffffffu;
        for (int i = 0; i < nw; i++) r &= red[i][lane];
        if (r != 0xffffffffu) atomicAnd(&valid[w], r);
    }
}

// ------------------------------------------------------------ dedup ------
constexpr unsigned long long EMPTY_SLOT = ~0ull;

// SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// h = golden gamma; h = mix64(h + word) over 64-bit key words; h = mix64(h ^ n_words).
__device__ __forceinline__ uint64_t key_hash(const uint32_t* key, int kw) {
    const int n64 = (kw + 1) / 2;
    uint64_t h = 0x9E3779B97F4A7C15ull;
    for (int w = 0; w < n64; w++) {
        const uint64_t lo = key[2 * w];
        const uint64_t hi = (2 * w + 1 < kw) ? key[2 * w + 1] : 0u;
        h = mix64(h + (lo | (hi << 32)));
    }
    return mix64(h ^ (uint64_t)n64);
}

__device__ __forceinline__ bool keys_equal(const uint32_t* a, const uint32_t* b, int kw) {
    for (int i = 0; i < kw; i++)
        if (a[i] != b[i]) return false;
    return true;
}

// Open addressing with linear probing; a slot holds (hash >> 32) << 32 | index,
// the index pointing into this batch's keys (bit 31 set) or the key pool.
__global__ void dedup_insert_kernel(DevDedup d, const uint32_t* keys, const uint32_t* valid, int64_t B,
                                    unsigned long long* hashes, uint8_t* is_new, unsigned long long* slot_of) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    const int kw = d.key_words;
    const bool val = (valid[s >> 5] >> (s & 31)) & 1u;
    uint8_t fresh = 0;
    unsigned long long where = EMPTY_SLOT;
    uint64_t h = 0;
    if (val) {
        const uint32_t* key = keys + s * kw;
        h = key_hash(key, kw);
        const unsigned long long tag = (h >> 32) << 32;
        const unsigned long long mine = tag | 0x80000000ull | (unsigned long long)s;
        uint64_t pos = h & (d.capacity - 1);
        bool done = false;
        for (uint32_t probe = 0; probe < d.max_probe; probe++) {
            const unsigned long long cur = atomicCAS(&d.slots[pos], EMPTY_SLOT, mine);
            if (cur == EMPTY_SLOT) {
                fresh = 1;
                where = pos;
                done = true;
                break;
            }
            if ((cur & 0xffffffff00000000ull) == tag) {
                const uint64_t idx = cur & 0x7fffffffull;
                const uint32_t* other = (cur & 0x80000000ull) ? keys + idx * kw : d.pool + idx * kw;
                if (keys_equal(key, other, kw)) {
                    done = true;
                    break;
                }
            }
            pos = (pos + 1) & (d.capacity - 1);
        }
        if (!done) atomicOr(d.status, 1u);
    }
    if (hashes) hashes[s] = h;
    if (is_new) is_new[s] = fresh;
    slot_of[s] = where;
}

// Move this batch's new keys into the pool and point their slots at it.
__global__ void dedup_commit_kernel(DevDedup d, const uint32_t* keys, int64_t B, const unsigned long long* slot_of) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    const unsigned long long pos = slot_of[s];
    if (pos == EMPTY_SLOT) return;
    const unsigned long long idx = atomicAdd(d.count, 1ull);
    if (idx >= d.pool_capacity) {  // cannot happen when the host checked capacity first
        atomicOr(d.status, 2u);
        d.slots[pos] = EMPTY_SLOT;
        return;
    }
    const int kw = d.key_words;
    for (int i = 0; i < kw; i++) d.pool[idx * kw + i] = keys[s * kw + i];
    d.slots[pos] = (d.slots[pos] & 0xffffffff00000000ull) | idx;
}

template <typename T>
cudaError_t forward_launch(const DevPlan& p, const float* V, int64_t ldv, void* act, float* loss, int64_t B,
                           cudaStream_t s) {
    cudaError_t e = prepare_tile_kernels<T>();
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((B + TILE - 1) / TILE);
    forward_kernel<T><<<grid, STEP_THREADS, stage_smem<T>(), s>>>(p, V, ldv, (T*)act, loss, B);
    return cudaGetLastError();
}

template <typename T>
cudaError_t backward_launch(const DevPlan& p, const float* V, int64_t ldv, const void* act, float* adj,
                            const float* grad_loss, float* gV, int64_t B, cudaStream_t s) {
    cudaError_t e = prepare_tile_kernels<T>();
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((B + TILE - 1) / TILE);
    backward_kernel<T><<<grid, STEP_THREADS, stage_smem<T>(), s>>>(p, V, ldv, (const T*)act, adj, grad_loss, gV, B);
    return cudaGetLastError();
}

template <typename T>
cudaError_t steps_launch(const DevPlan& p, const OptParams& o, float* V, float* m, float* v, int64_t ldv, void* act,
                         float* adj, float* loss, int t0, int n_steps, int64_t B, cudaStream_t s) {
    cudaError_t e = prepare_tile_kernels<T>();
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((B + TILE - 1) / TILE);
    const double p1 = std::pow((double)o.b1, (double)(t0 - 1)), p2 = std::pow((double)o.b2, (double)(t0 - 1));
    steps_kernel<T><<<grid, STEP_THREADS, stage_smem<T>(), s>>>(p, o, V, m, v, ldv, (T*)act, adj, loss, p1, p2,
                                                                n_steps, B);
    return cudaGetLastError();
}

}  // namespace

// ------------------------------------------------------------ launchers --
cudaError_t launch_init_normal(const DevPlan& p, uint64_t seed, uint32_t round, float scale, float* V, int64_t ldv,
                               int64_t B, cudaStream_t s) {
    const int64_t n = (int64_t)p.n_pi * B;
    if (n == 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 148 * 32);
    init_normal_kernel<<<grid, 256, 0, s>>>(p.n_pi, seed, round, scale, V, ldv, B);
    return cudaGetLastError();
}

cudaError_t launch_forward(const DevPlan& p, int act_type, const float* V, int64_t ldv, void* act, float* loss,
                           int64_t B, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    switch (act_type) {
    case ACT_F32: return forward_launch<float>(p, V, ldv, act, loss, B, s);
    case ACT_BF16: return forward_launch<__nv_bfloat16>(p, V, ldv, act, loss, B, s);
    default: return forward_launch<__half>(p, V, ldv, act, loss, B, s);
    }
}

cudaError_t launch_backward(const DevPlan& p, int act_type, const float* V, int64_t ldv, const void* act, float* adj,
                            const float* grad_loss, float* gV, int64_t B, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    switch (act_type) {
    case ACT_F32: return backward_launch<float>(p, V, ldv, act, adj, grad_loss, gV, B, s);
    case ACT_BF16: return backward_launch<__nv_bfloat16>(p, V, ldv, act, adj, grad_loss, gV, B, s);
    default: return backward_launch<__half>(p, V, ldv, act, adj, grad_loss, gV, B, s);
    }
}

cudaError_t launch_steps(const DevPlan& p, int act_type, const OptParams& o, float* V, float* m, float* v, int64_t ldv,
                         void* act, float* adj, float* loss, int t0, int n_steps, int64_t B, cudaStream_t s) {
    if (B == 0 || n_steps <= 0) return cudaSuccess;
    switch (act_type) {
    case ACT_F32: return steps_launch<float>(p, o, V, m, v, ldv, act, adj, loss, t0, n_steps, B, s);
    case ACT_BF16: return steps_launch<__nv_bfloat16>(p, o, V, m, v, ldv, act, adj, loss, t0, n_steps, B, s);
    default: return steps_launch<__half>(p, o, V, m, v, ldv, act, adj, loss, t0, n_steps, B, s);
    }
}

cudaError_t launch_opt_update(const DevPlan& p, const OptParams& o, float* V, float* m, float* v, const float* gV,
                              int64_t ldv, int t, int64_t B, cudaStream_t s) {
    const int64_t n = (int64_t)p.n_cone_pi * B;
    if (n == 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 148 * 32);
    const double p1 = std::pow((double)o.b1, (double)t), p2 = std::pow((double)o.b2, (double)t);
    opt_update_kernel<<<grid, 256, 0, s>>>(p, o, V, m, v, gV, ldv, p1, p2, B);
    return cudaGetLastError();
}

cudaError_t launch_threshold(const DevPlan& p, const float* V, int64_t ldv, uint32_t* node_bits, int64_t ldw,
                             uint32_t* keys, int64_t B, cudaStream_t s) {
    if (B == 0 || p.n_pi == 0) return cudaSuccess;
    dim3 grid((unsigned)((B + 31) / 32), (unsigned)((p.n_pi + 31) / 32));
    threshold_kernel<<<grid, dim3(32, 32), 0, s>>>(V, ldv, p.n_pi, node_bits, ldw, keys, p.key_words, B);
    return cudaGetLastError();
}

cudaError_t launch_hard_eval(const DevPlan& p, uint32_t* node_bits, int64_t ldw, int64_t B, cudaStream_t s) {
    const int64_t W = (B + 31) / 32;
    if (W == 0 || p.n_flev == 0) return cudaSuccess;
    hard_eval_kernel<8><<<(unsigned)((W + 7) / 8), 512, 0, s>>>(p, node_bits, ldw, W);
    return cudaGetLastError();
}

cudaError_t launch_cnf_check(const DevPlan& p, const uint32_t* node_bits, int64_t ldw, uint32_t* valid, int64_t B,
                             cudaStream_t s) {
    const int64_t W = (B + 31) / 32;
    if (W == 0) return cudaSuccess;
    valid_init_kernel<<<(unsigned)((W + 255) / 256), 256, 0, s>>>(valid, W, B);
    if (p.n_clauses > 0) {
        dim3 grid((unsigned)((W + 31) / 32), (unsigned)((p.n_clauses + CLAUSES_PER_CTA - 1) / CLAUSES_PER_CTA));
        cnf_check_kernel<<<grid, 256, 0, s>>>(p, node_bits, ldw, valid, W);
    }
    return cudaGetLastError();
}

cudaError_t launch_dedup_clear(DevDedup& d, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(d.slots, 0xff, d.capacity * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(d.count, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(d.status, 0, sizeof(unsigned int), s);
}

cudaError_t launch_dedup_insert(DevDedup& d, const uint32_t* keys, const uint32_t* valid, int64_t B,
                                unsigned long long* hashes, uint8_t* is_new, unsigned long long* slot_of,
                                cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((B + 255) / 256);
    dedup_insert_kernel<<<grid, 256, 0, s>>>(d, keys, valid, B, hashes, is_new, slot_of);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dedup_commit_kernel<<<grid, 256, 0, s>>>(d, keys, B, slot_of);
    return cudaGetLastError();
}

}  // namespace sat
