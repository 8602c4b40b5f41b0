// Kernels of the sampling loop around the step kernels (sm_103a): the Gaussian
// initialisation of V, early-exit retire/restart, the hard threshold, the Boolean pass
// over every gate, the check of the original clauses and the device hash set of
// distinct solutions.  Layout: V rows are primary inputs over the batch; node bits are
// rows of 32-sample words (word w holds samples 32w .. 32w + 31); keys are a sample's
// primary-input bits, key_words 32-bit words per sample.
#include <algorithm>
#include <cstdint>

#include "device.hpp"
#include "philox.cuh"

namespace sat {
namespace {

constexpr unsigned FULL = 0xffffffffu;

// ------------------------------------------------------------ init -------
// V[r][b] = scale * z, z the (b mod 4)-th normal of group c = b / 4 of row r (normal4).
// One thread per group of four samples (coalesced within a row), rows on y, both
// grid-stride; 16-byte stores where the group is whole and aligned.
__global__ void init_normal_kernel(int32_t n_pi, uint64_t seed, uint32_t round, float scale, float* V, int64_t ldv,
                                   int64_t B) {
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const int64_t groups = (B + 3) / 4;
    for (int64_t r = blockIdx.y; r < n_pi; r += gridDim.y)
        for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < groups;
             c += (int64_t)gridDim.x * blockDim.x) {
            const float4 z = normal4((uint32_t)c, (uint32_t)r, round, key);
            float* out = V + r * ldv + 4 * c;
            const float4 x = make_float4(scale * z.x, scale * z.y, scale * z.z, scale * z.w);
            if (4 * c + 3 < B && ((uintptr_t)out & 15u) == 0) {
                *reinterpret_cast<float4*>(out) = x;
            } else {
                const float xs[4] = {x.x, x.y, x.z, x.w};
                for (int k = 0; k < 4 && 4 * c + k < B; k++) out[k] = xs[k];
            }
        }
}

// ------------------------------------------------------- early exit -----
// One thread per sample; a warp's ballot is one restart word (32 samples).
__global__ void retire_kernel(const uint32_t* valid, int32_t* age, uint32_t* restart, int k, int max_age, int64_t B) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool r = false;
    if (b < B) {
        const int a = age[b];
        r = ((valid[b >> 5] >> (b & 31)) & 1u) != 0u || a + k >= max_age;
        age[b] = r ? 0 : a + k;
    }
    const unsigned w = __ballot_sync(0xffffffffu, r);
    if ((threadIdx.x & 31) == 0 && b < B) restart[b >> 5] = w;
}

// Samples on x (coalesced within a row), rows on y (grid-stride).
__global__ void restart_kernel(int32_t n_pi, const uint32_t* restart, uint64_t seed, uint32_t round, float scale,
                               const float* src, int64_t lds, float* V, float* m, float* v, int64_t ldv, int64_t B) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B || ((restart[b >> 5] >> (b & 31)) & 1u) == 0u) return;
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    for (int64_t r = blockIdx.y; r < n_pi; r += gridDim.y) {
        float x;
        if (src) {
            x = src[r * lds + b];
        } else {
            const float4 z = normal4((uint32_t)(b >> 2), (uint32_t)r, round, key);  // what init draws for b
            const int k = (int)(b & 3);
            x = scale * (k == 0 ? z.x : k == 1 ? z.y : k == 2 ? z.z : z.w);
        }
        V[r * ldv + b] = x;
        m[r * ldv + b] = 0.0f;
        v[r * ldv + b] = 0.0f;
    }
}

// ---------------------------------------------------- verification -------
// Threshold (bit = V > 0) in two passes.  Bits: one warp per (input row, segment of 32
// words = 1,024 samples); lane j loads V[r][b0 + 32k + j] for k = 0..31 (32 coalesced
// 128-byte loads in flight, 4 KB contiguous per row), the ballot of load k is word k of the
// row, and lane k stores it (one coalesced store of the segment's words).
__global__ void __launch_bounds__(256) threshold_bits_kernel(const float* V, int64_t ldv, int32_t n_pi, uint32_t* bits,
                                                             int64_t ldw, int64_t B) {
    const int lane = threadIdx.x & 31;
    const int64_t W = (B + 31) / 32, nseg = (W + 31) / 32;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nseg * n_pi; t += nwarps) {
        const int64_t r = t / nseg, seg = t - r * nseg;
        const float* row = V + r * ldv;
        const int64_t b0 = seg * 1024 + lane;
        float x[32];
#pragma unroll
        for (int k = 0; k < 32; k++) x[k] = b0 + 32 * k < B ? row[b0 + 32 * k] : 0.0f;
        uint32_t mine = 0;
#pragma unroll
        for (int k = 0; k < 32; k++) {
            const unsigned wb = __ballot_sync(FULL, x[k] > 0.0f);
            if (lane == k) mine = wb;
        }
        if (seg * 32 + lane < W) bits[r * ldw + seg * 32 + lane] = mine;
    }
}

// Keys: one warp per (word w, block g of 32 inputs); lane i holds word w of input row
// 32g + i, and the ballot of bit j over the lanes is sample 32w + j's key word g (a 32 x 32
// bit transpose), kept by lane j.
__global__ void __launch_bounds__(256) threshold_keys_kernel(const uint32_t* bits, int64_t ldw, int32_t n_pi,
                                                             uint32_t* keys, int32_t kw, int64_t B) {
    const int lane = threadIdx.x & 31;
    const int64_t W = (B + 31) / 32, ng = (n_pi + 31) / 32;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < W * ng; t += nwarps) {
        const int64_t g = t / W, w = t - g * W;
        const int64_t r = g * 32 + lane;
        const uint32_t word = r < n_pi ? bits[r * ldw + w] : 0u;
        uint32_t key = 0;
#pragma unroll
        for (int j = 0; j < 32; j++) {
            const unsigned kb = __ballot_sync(FULL, (word >> j) & 1u);
            if (lane == j) key = kb;
        }
        const int64_t b = w * 32 + lane;
        if (b < B) keys[b * kw + g] = key;
    }
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

// Move this batch's new keys into the pool and point their slots at it.  Pool indices are
// taken one atomic add per warp (the warp's new keys, in lane order).
__global__ void dedup_commit_kernel(DevDedup d, const uint32_t* keys, int64_t B, const unsigned long long* slot_of) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long pos = s < B ? slot_of[s] : EMPTY_SLOT;
    const bool mine = pos != EMPTY_SLOT;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned ballot = __ballot_sync(0xffffffffu, mine);
    if (ballot == 0u) return;
    const int leader = __ffs(ballot) - 1;
    unsigned long long base = 0;
    if ((int)lane == leader) base = atomicAdd(d.count, (unsigned long long)__popc(ballot));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (!mine) return;
    const unsigned long long idx = base + (unsigned long long)__popc(ballot & ((1u << lane) - 1u));
    if (idx >= d.pool_capacity) {  // cannot happen when the host checked capacity first
        atomicOr(d.status, 2u);
        d.slots[pos] = EMPTY_SLOT;
        return;
    }
    const int kw = d.key_words;
    for (int i = 0; i < kw; i++) d.pool[idx * kw + i] = keys[s * kw + i];
    d.slots[pos] = (d.slots[pos] & 0xffffffff00000000ull) | idx;
}

// Diagnostic: for every point of the Box-Muller angle grid, the signs of sincospif's sine and
// cosine (bm_angle, as normal4 computes them) against bm_angle_signs; counts disagreements.
__global__ void angle_signs_diag_kernel(unsigned* mismatches) {
    unsigned bad = 0;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < (1u << 24); k += gridDim.x * blockDim.x) {
        float sn, cs;
        bm_angle(k << 8, &sn, &cs);
        int dc, ds;
        bm_angle_signs(k << 8, &dc, &ds);
        const int sc = cs > 0.0f ? 1 : cs < 0.0f ? -1 : 0, ss = sn > 0.0f ? 1 : sn < 0.0f ? -1 : 0;
        bad += (sc != dc) + (ss != ds);
    }
    if (bad) atomicAdd(mismatches, bad);
}

}  // namespace

cudaError_t launch_angle_signs_diag(unsigned* mismatches, cudaStream_t s) {
    angle_signs_diag_kernel<<<1024, 256, 0, s>>>(mismatches);
    return cudaGetLastError();
}

cudaError_t launch_init_normal(const DevPlan& p, uint64_t seed, uint32_t round, float scale, float* V, int64_t ldv,
                               int64_t B, cudaStream_t s) {
    const int64_t n = (int64_t)p.n_pi * B;
    if (n == 0) return cudaSuccess;
    const int64_t groups = (B + 3) / 4;
    const dim3 grid((unsigned)std::min<int64_t>((groups + 255) / 256, 1024),
                    (unsigned)std::min<int64_t>(p.n_pi, 65535));
    init_normal_kernel<<<grid, 256, 0, s>>>(p.n_pi, seed, round, scale, V, ldv, B);
    return cudaGetLastError();
}

cudaError_t launch_retire(const uint32_t* valid, int32_t* age, uint32_t* restart, int k, int max_age, int64_t B,
                          cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    retire_kernel<<<(unsigned)((B + 255) / 256), 256, 0, s>>>(valid, age, restart, k, max_age, B);
    return cudaGetLastError();
}

cudaError_t launch_restart(const DevPlan& p, const uint32_t* restart, uint64_t seed, uint32_t round, float scale,
                           const float* src, int64_t lds, float* V, float* m, float* v, int64_t ldv, int64_t B,
                           cudaStream_t s) {
    if (B == 0 || p.n_pi == 0) return cudaSuccess;
    const dim3 grid((unsigned)((B + 255) / 256), (unsigned)std::min<int64_t>(p.n_pi, 256));
    restart_kernel<<<grid, 256, 0, s>>>(p.n_pi, restart, seed, round, scale, src, lds, V, m, v, ldv, B);
    return cudaGetLastError();
}

cudaError_t launch_threshold(const DevPlan& p, const float* V, int64_t ldv, uint32_t* node_bits, int64_t ldw,
                             uint32_t* keys, int64_t B, cudaStream_t s) {
    if (B == 0 || p.n_pi == 0) return cudaSuccess;
    const int64_t W = (B + 31) / 32;
    const int64_t bit_tasks = ((W + 31) / 32) * p.n_pi, key_tasks = W * ((p.n_pi + 31) / 32);  // one per warp
    threshold_bits_kernel<<<(unsigned)std::min<int64_t>((bit_tasks + 7) / 8, 148 * 16), 256, 0, s>>>(
        V, ldv, p.n_pi, node_bits, ldw, B);
    threshold_keys_kernel<<<(unsigned)std::min<int64_t>((key_tasks + 7) / 8, 148 * 16), 256, 0, s>>>(
        node_bits, ldw, p.n_pi, keys, p.key_words, B);
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
