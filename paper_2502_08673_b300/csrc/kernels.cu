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

#include "device.hpp"

namespace sat {
namespace {

constexpr int TILE = 32;
constexpr int STEP_THREADS = 512;
constexpr int UNROLL = 4;

template <typename T> struct ActIO;
template <> struct ActIO<float> {
    static __device__ __forceinline__ float ld(const float* p) { return *p; }
    static __device__ __forceinline__ void st(float* p, float x) { *p = x; }
};
template <> struct ActIO<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float x) { *p = __float2bfloat16_rn(x); }
};
template <> struct ActIO<__half> {
    static __device__ __forceinline__ float ld(const __half* p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half* p, float x) { *p = __float2half_rn(x); }
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

struct TileCtx {
    int lane, warp, nw;
    int64_t b;     // sample index of this lane
    bool ok;       // b < B
};

__device__ __forceinline__ TileCtx tile_ctx(int64_t B) {
    TileCtx c;
    c.lane = threadIdx.x & 31;
    c.warp = threadIdx.x >> 5;
    c.nw = blockDim.x >> 5;
    c.b = (int64_t)blockIdx.x * TILE + c.lane;
    c.ok = c.b < B;
    return c;
}

// Forward pass of one tile: P = sigmoid(V) for cone inputs, then every cone level.
template <typename T>
__device__ void tile_forward(const DevPlan& p, const float* __restrict__ V, int64_t ldv, T* act, int64_t lda,
                             const TileCtx& c) {
    for (int i = c.warp; i < p.n_cone_pi; i += c.nw) {
        float P = 0.5f;
        if (c.ok) P = sigmoidf_(V[(int64_t)p.cone_pi_row[i] * ldv + c.b]);
        ActIO<T>::st(act + (int64_t)i * lda + c.b, P);
    }
    __syncthreads();
    for (int l = 1; l <= p.n_clev; l++) {
        const int lo = p.c_level_off[l], hi = p.c_level_off[l + 1];
        for (int g0 = lo + c.warp; g0 < hi; g0 += UNROLL * c.nw) {
            int2 gm[UNROLL];
            float x[UNROLL], y[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; u++) {
                const int g = g0 + u * c.nw;
                gm[u] = g < hi ? __ldg(&p.c_gate[g - p.n_cone_pi]) : make_int2(0, 0);
            }
#pragma unroll
            for (int u = 0; u < UNROLL; u++) {
                const int g = g0 + u * c.nw;
                if (g < hi) {
                    x[u] = ActIO<T>::ld(act + (int64_t)(gm[u].x & 0x0FFFFFFF) * lda + c.b);
                    y[u] = ActIO<T>::ld(act + (int64_t)gm[u].y * lda + c.b);
                }
            }
#pragma unroll
            for (int u = 0; u < UNROLL; u++) {
                const int g = g0 + u * c.nw;
                if (g < hi) ActIO<T>::st(act + (int64_t)g * lda + c.b, gate_eval((uint32_t)gm[u].x >> 28, x[u], y[u]));
            }
        }
        __syncthreads();
    }
}

// Per-sample loss sum_j (Y_j - T_j)^2, FP32, fixed order (warp-strided partials, then warp order).
template <typename T>
__device__ void tile_loss(const DevPlan& p, const T* act, int64_t lda, float* loss, const TileCtx& c) {
    __shared__ float part[STEP_THREADS / 32][32];
    float acc = 0.0f;
    for (int j = c.warp; j < p.n_out; j += c.nw) {
        const float e = ActIO<T>::ld(act + (int64_t)p.c_out_node[j] * lda + c.b) - p.out_target[j];
        acc = fmaf(e, e, acc);
    }
    part[c.warp][c.lane] = acc;
    __syncthreads();
    if (c.warp == 0) {
        float s = 0.0f;
        for (int w = 0; w < c.nw; w++) s += part[w][c.lane];
        if (c.ok) loss[c.b] = s;
    }
    __syncthreads();
}

// Adjoint of cone node u: output seeds and fan-out contributions in CSR order.
template <typename T>
__device__ __forceinline__ float node_adjoint(const DevPlan& p, int u, const T* act, const float* adj, int64_t lda,
                                              float seed_scale, const TileCtx& c) {
    const int64_t e0 = p.fo_off[u], e1 = p.fo_off[u + 1];
    float acc = 0.0f;
    for (int64_t e = e0; e < e1; e++) {
        const int4 E = __ldg(&p.fo_edge[e]);
        if (E.x < 0) {
            const float y = ActIO<T>::ld(act + (int64_t)u * lda + c.b);
            acc = fmaf(2.0f * seed_scale, y - (float)E.y, acc);
        } else {
            const float ga = adj[(int64_t)E.x * lda + c.b];
            const float s = ActIO<T>::ld(act + (int64_t)E.y * lda + c.b);
            acc = fmaf(ga, fmaf((float)E.w, s, (float)E.z), acc);
        }
    }
    return acc;
}

// Backward pass of one tile over levels n_clev..1; then the input level, where
// the adjoint of P becomes dL/dV = Pbar * P (1 - P) and is either stored (gV)
// or applied by the optimiser.
template <typename T, bool UPDATE>
__device__ void tile_backward(const DevPlan& p, const OptParams& o, float* V, float* m, float* v, float* gV,
                              int64_t ldv, const T* act, float* adj, int64_t lda, const float* grad_loss, int t,
                              const TileCtx& c) {
    const float seed_scale = (grad_loss != nullptr && c.ok) ? grad_loss[c.b] : 1.0f;
    for (int l = p.n_clev; l >= 1; l--) {
        const int lo = p.c_level_off[l], hi = p.c_level_off[l + 1];
        for (int u = lo + c.warp; u < hi; u += c.nw)
            adj[(int64_t)u * lda + c.b] = node_adjoint<T>(p, u, act, adj, lda, seed_scale, c);
        __syncthreads();
    }
    float step_size = 0.0f, bc2s = 1.0f;
    if (UPDATE && o.opt == 0) {
        const double bc1 = 1.0 - pow((double)o.b1, (double)t);
        const double bc2 = 1.0 - pow((double)o.b2, (double)t);
        step_size = (float)((double)o.lr / bc1);
        bc2s = (float)sqrt(bc2);
    }
    for (int i = c.warp; i < p.n_cone_pi; i += c.nw) {
        const float pbar = node_adjoint<T>(p, i, act, adj, lda, seed_scale, c);
        if (!c.ok) continue;
        const int64_t r = (int64_t)p.cone_pi_row[i] * ldv + c.b;
        const float P = sigmoidf_(V[r]);
        const float g = pbar * P * (1.0f - P);
        if (!UPDATE) {
            gV[r] = g;
        } else if (o.opt == 1) {
            V[r] = fmaf(-o.lr, g, V[r]);
        } else {
            float mm = m[r], vv = v[r];
            mm = fmaf(1.0f - o.b1, g - mm, mm);
            vv = fmaf(o.b2, vv, (1.0f - o.b2) * g * g);
            m[r] = mm;
            v[r] = vv;
            const float denom = sqrtf(vv) / bc2s + o.eps;
            V[r] = V[r] - step_size * (mm / denom);
        }
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(STEP_THREADS) forward_kernel(DevPlan p, const float* V, int64_t ldv, T* act,
                                                               int64_t lda, float* loss, int64_t B) {
    const TileCtx c = tile_ctx(B);
    tile_forward<T>(p, V, ldv, act, lda, c);
    if (loss) tile_loss<T>(p, act, lda, loss, c);
}

template <typename T>
__global__ void __launch_bounds__(STEP_THREADS) backward_kernel(DevPlan p, const float* V, int64_t ldv, const T* act,
                                                                int64_t lda, float* adj, const float* grad_loss,
                                                                float* gV, int64_t B) {
    const TileCtx c = tile_ctx(B);
    OptParams o;
    tile_backward<T, false>(p, o, const_cast<float*>(V), nullptr, nullptr, gV, ldv, act, adj, lda, grad_loss, 0, c);
}

// The fused hot loop: n_steps x (forward, loss, adjoint, update) for one tile.
template <typename T>
__global__ void __launch_bounds__(STEP_THREADS) steps_kernel(DevPlan p, OptParams o, float* V, float* m, float* v,
                                                             int64_t ldv, T* act, float* adj, int64_t lda,
                                                             float* loss, int t0, int n_steps, int64_t B) {
    const TileCtx c = tile_ctx(B);
    for (int s = 0; s < n_steps; s++) {
        tile_forward<T>(p, V, ldv, act, lda, c);
        if (loss && s == n_steps - 1) tile_loss<T>(p, act, lda, loss, c);
        tile_backward<T, true>(p, o, V, m, v, nullptr, ldv, act, adj, lda, nullptr, t0 + s, c);
    }
}

__global__ void opt_update_kernel(DevPlan p, OptParams o, float* V, float* m, float* v, const float* gV, int64_t ldv,
                                  int t, int64_t B) {
    const int64_t n = (int64_t)p.n_cone_pi * B;
    const double bc1 = 1.0 - pow((double)o.b1, (double)t);
    const double bc2 = 1.0 - pow((double)o.b2, (double)t);
    const float step_size = (float)((double)o.lr / bc1), bc2s = (float)sqrt(bc2);
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
cudaError_t steps_launch(const DevPlan& p, const OptParams& o, float* V, float* m, float* v, int64_t ldv, void* act,
                         float* adj, int64_t lda, float* loss, int t0, int n_steps, int64_t B, cudaStream_t s) {
    const unsigned grid = (unsigned)((B + TILE - 1) / TILE);
    steps_kernel<T><<<grid, STEP_THREADS, 0, s>>>(p, o, V, m, v, ldv, (T*)act, adj, lda, loss, t0, n_steps, B);
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

cudaError_t launch_forward(const DevPlan& p, int act_type, const float* V, int64_t ldv, void* act, int64_t lda,
                           float* loss, int64_t B, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((B + TILE - 1) / TILE);
    switch (act_type) {
    case ACT_F32: forward_kernel<float><<<grid, STEP_THREADS, 0, s>>>(p, V, ldv, (float*)act, lda, loss, B); break;
    case ACT_BF16: forward_kernel<__nv_bfloat16><<<grid, STEP_THREADS, 0, s>>>(p, V, ldv, (__nv_bfloat16*)act, lda, loss, B); break;
    default: forward_kernel<__half><<<grid, STEP_THREADS, 0, s>>>(p, V, ldv, (__half*)act, lda, loss, B); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_backward(const DevPlan& p, int act_type, const float* V, int64_t ldv, const void* act, int64_t lda,
                            float* adj, const float* grad_loss, float* gV, int64_t B, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((B + TILE - 1) / TILE);
    switch (act_type) {
    case ACT_F32: backward_kernel<float><<<grid, STEP_THREADS, 0, s>>>(p, V, ldv, (const float*)act, lda, adj, grad_loss, gV, B); break;
    case ACT_BF16: backward_kernel<__nv_bfloat16><<<grid, STEP_THREADS, 0, s>>>(p, V, ldv, (const __nv_bfloat16*)act, lda, adj, grad_loss, gV, B); break;
    default: backward_kernel<__half><<<grid, STEP_THREADS, 0, s>>>(p, V, ldv, (const __half*)act, lda, adj, grad_loss, gV, B); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_steps(const DevPlan& p, int act_type, const OptParams& o, float* V, float* m, float* v, int64_t ldv,
                         void* act, float* adj, int64_t lda, float* loss, int t0, int n_steps, int64_t B,
                         cudaStream_t s) {
    if (B == 0 || n_steps <= 0) return cudaSuccess;
    switch (act_type) {
    case ACT_F32: return steps_launch<float>(p, o, V, m, v, ldv, act, adj, lda, loss, t0, n_steps, B, s);
    case ACT_BF16: return steps_launch<__nv_bfloat16>(p, o, V, m, v, ldv, act, adj, lda, loss, t0, n_steps, B, s);
    default: return steps_launch<__half>(p, o, V, m, v, ldv, act, adj, lda, loss, t0, n_steps, B, s);
    }
}

cudaError_t launch_opt_update(const DevPlan& p, const OptParams& o, float* V, float* m, float* v, const float* gV,
                              int64_t ldv, int t, int64_t B, cudaStream_t s) {
    const int64_t n = (int64_t)p.n_cone_pi * B;
    if (n == 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 148 * 32);
    opt_update_kernel<<<grid, 256, 0, s>>>(p, o, V, m, v, gV, ldv, t, B);
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
