// CUDA kernels of the sampler's hot path (sm_103a).
//
// Layout: every per-sample quantity is stored node-major with the batch
// contiguous ("SoA"): row r of V, m, v, gV is primary input r over the batch.
// The per-node scratch (act, adj) is tile-major: a CTA owns a tile of TILE
// samples (VEC consecutive samples per lane) and its contiguous blocks of
// [rows][TILE] (act rows per the act layout, adj rows per the adjoint ring),
// and walks the levels of the circuit.  Samples are
// independent, so the only synchronisation is __syncthreads between levels.
//
// Relaxation (Table 1): with input negation x -> 1 - x folded in, every
// 2-input gate is a bilinear form y = k0 + k1 a + k2 b + k3 a b (AND: a b;
// OR: a + b - a b; XOR: a + b - 2 a b); embedding P = sigmoid(V) (Eq. 5); loss
// sum_j (Y_j - T_j)^2 (Eq. 7); the adjoint is the chain rule of Eq. 8 in
// gather form (each node sums, in a fixed order, the contributions of its
// fan-out edges); the update is Eq. 9 (GD) or Adam in PyTorch's formulation.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>
#include <type_traits>
#include <cmath>

#include "device.hpp"
#include "relax.cuh"
#include "tmap.hpp"

namespace sat {
namespace {

#ifndef SAT_VEC
#define SAT_VEC 4
#endif
constexpr int VEC = SAT_VEC;           // consecutive samples per lane
constexpr int TILE = 32 * VEC;         // samples per CTA
static_assert(TILE == SAT_TILE_SAMPLES, "tile width must match the ABI");
// Threads of a step-kernel CTA: 20 warps with FP32 activations, 24 with 16-bit ones
// (their smaller staging slots leave room; measured best for each).
template <typename T>
__host__ __device__ constexpr int step_threads() { return sizeof(T) == 4 ? 640 : 768; }
static_assert(step_threads<float>() / 32 == loss_partials<float>() &&
                  step_threads<__half>() / 32 == loss_partials<__half>(),
              "the tiled loss sums one partial per warp");
constexpr int UBATCH = 2;              // input rows per warp in the input-level passes
constexpr unsigned FULL = 0xffffffffu;

// VEC consecutive samples of one row, in registers.
struct VF {
    float v[VEC];
};

__device__ __forceinline__ VF vf_fill(float x) {
    VF r;
#pragma unroll
    for (int q = 0; q < VEC; q++) r.v[q] = x;
    return r;
}

template <typename T> struct ActIO;
template <> struct ActIO<float> {
    static __device__ __forceinline__ VF ld(const float* p) {
        VF r;
        if constexpr (VEC == 4) {
            const float4 q = *reinterpret_cast<const float4*>(p);
            r.v[0] = q.x; r.v[1] = q.y; r.v[2] = q.z; r.v[3] = q.w;
        } else {
            const float2 q = *reinterpret_cast<const float2*>(p);
            r.v[0] = q.x; r.v[1] = q.y;
        }
        return r;
    }
    // L2-only load (bypasses L1): for rows another SM may have written
    static __device__ __forceinline__ VF ldcg(const float* p) {
        VF r;
        if constexpr (VEC == 4) {
            const float4 q = __ldcg(reinterpret_cast<const float4*>(p));
            r.v[0] = q.x; r.v[1] = q.y; r.v[2] = q.z; r.v[3] = q.w;
        } else {
            const float2 q = __ldcg(reinterpret_cast<const float2*>(p));
            r.v[0] = q.x; r.v[1] = q.y;
        }
        return r;
    }
    static __device__ __forceinline__ void st(float* p, const VF& x) {
        if constexpr (VEC == 4) *reinterpret_cast<float4*>(p) = make_float4(x.v[0], x.v[1], x.v[2], x.v[3]);
        else *reinterpret_cast<float2*>(p) = make_float2(x.v[0], x.v[1]);
    }
};
// 16-bit storage: a lane's VEC = 4 values are one 8-byte word (two 16-bit pairs), moved
// with one load or store; ldcg reads them through L2 only.
template <typename H, typename H2>
struct ActIO16 {
    static_assert(VEC == 4, "one 8-byte word per lane");
    static __device__ __forceinline__ VF unpack(uint2 u, float2 (*cvt)(H2)) {
        const float2 a = cvt(*reinterpret_cast<const H2*>(&u.x)), b = cvt(*reinterpret_cast<const H2*>(&u.y));
        VF r;
        r.v[0] = a.x; r.v[1] = a.y; r.v[2] = b.x; r.v[3] = b.y;
        return r;
    }
    static __device__ __forceinline__ uint2 pack(const VF& x, H2 (*cvt)(float2)) {
        const H2 a = cvt(make_float2(x.v[0], x.v[1])), b = cvt(make_float2(x.v[2], x.v[3]));
        return make_uint2(*reinterpret_cast<const unsigned*>(&a), *reinterpret_cast<const unsigned*>(&b));
    }
};
template <> struct ActIO<__nv_bfloat16> {
    using IO = ActIO16<__nv_bfloat16, __nv_bfloat162>;
    static __device__ __forceinline__ VF ld(const __nv_bfloat16* p) {
        return IO::unpack(*reinterpret_cast<const uint2*>(p), __bfloat1622float2);
    }
    static __device__ __forceinline__ VF ldcg(const __nv_bfloat16* p) {
        return IO::unpack(__ldcg(reinterpret_cast<const uint2*>(p)), __bfloat1622float2);
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, const VF& x) {
        *reinterpret_cast<uint2*>(p) = IO::pack(x, __float22bfloat162_rn);
    }
};
template <> struct ActIO<__half> {
    using IO = ActIO16<__half, __half2>;
    static __device__ __forceinline__ VF ld(const __half* p) {
        return IO::unpack(*reinterpret_cast<const uint2*>(p), __half22float2);
    }
    static __device__ __forceinline__ VF ldcg(const __half* p) {
        return IO::unpack(__ldcg(reinterpret_cast<const uint2*>(p)), __half22float2);
    }
    static __device__ __forceinline__ void st(__half* p, const VF& x) {
        *reinterpret_cast<uint2*>(p) = IO::pack(x, __float22half2_rn);
    }
};



// A tile is processed by one CTA, or (split mode) by the two CTAs of a
// thread-block cluster, which divide every level's rows between their warps
// and meet at cluster barriers.  vw / nvw number the warps across the cluster.
struct TileCtx {
    int lane, warp, nw;
    int vw, nvw;    // work distribution: this warp among all warps serving the tile
    int rank;       // CTA within the cluster (0 outside split mode)
    int tile;       // tile index (samples tile*TILE .. tile*TILE+TILE-1)
    bool split;
    int64_t b;      // first of this lane's VEC samples
    int nvalid;     // how many of them are < B
};

__device__ __forceinline__ TileCtx tile_ctx(int64_t B, int tile0 = 0, bool split = false) {
    TileCtx c;
    c.lane = threadIdx.x & 31;
    c.warp = threadIdx.x >> 5;
    c.nw = blockDim.x >> 5;
    c.split = split;
    c.rank = split ? (int)(blockIdx.x & 1u) : 0;
    c.tile = tile0 + (int)(split ? blockIdx.x >> 1 : blockIdx.x);
    c.vw = c.rank * c.nw + c.warp;
    c.nvw = (split ? 2 : 1) * c.nw;
    c.b = (int64_t)c.tile * TILE + c.lane * VEC;
    const int64_t rem = B - c.b;
    c.nvalid = rem <= 0 ? 0 : (rem >= VEC ? VEC : (int)rem);
    return c;
}

// Element offset of this lane's samples in row `row` of a tile's [rows][TILE] block.
__device__ __forceinline__ uint32_t at(int row, const TileCtx& c) {
    return (uint32_t)row * TILE + (uint32_t)(c.lane * VEC);
}

// Barrier between levels: the CTA, or both CTAs of a split tile (release /
// acquire at cluster scope, so rows written by either CTA are visible after it).
__device__ __forceinline__ void level_sync(const TileCtx& c) {
    if (c.split)
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    else
        __syncthreads();
}


// Per-sample corrections of this lane's samples: step t, plus age[b] when
// samples restart at different steps (early exit), else the same t for all.
struct AdamCorr {
    float step[VEC], bc2s[VEC];
};
__device__ __forceinline__ AdamCorr adam_corr(const OptParams& o, const int32_t* age, int t, const TileCtx& c) {
    AdamCorr a;
    if (age == nullptr) {
        float st, bc;
        adam_bias(o, t, st, bc);
#pragma unroll
        for (int q = 0; q < VEC; q++) {
            a.step[q] = st;
            a.bc2s[q] = bc;
        }
    } else {
#pragma unroll
        for (int q = 0; q < VEC; q++) adam_bias(o, t + (q < c.nvalid ? __ldg(age + c.b + q) : 0), a.step[q], a.bc2s[q]);
    }
    return a;
}

// ------------------------------------------------------ async row copies --
// Rows of a tile's scratch block are staged into shared memory by the TMA
// engine: a chunk's rows come as tile::gather4 loads (four arbitrary rows per
// instruction through a 2-D tensor map over all tiles' rows, box = one row),
// completion counted in bytes on an mbarrier.  Each warp owns NSLOT slots and
// keeps NSLOT-1 chunks in flight while it computes on the oldest one.  Every mbarrier wait is
// bounded: on expiry the kernel records STATUS_WAIT_TIMEOUT in the plan's
// status word and carries on (results are then invalid, the GPU is not hung).
#ifndef SAT_CHUNK
#define SAT_CHUNK 4
#endif
constexpr int CHUNK = SAT_CHUNK;  // gates (forward) or fan-out edges (adjoint) per chunk
constexpr int NSLOT = 2;   // pipeline depth per warp (gathers land one chunk ahead: 93% of waits succeed at once)
static_assert(CHUNK == 4, "a chunk is one tile::gather4 load (4 rows) per operand");
constexpr unsigned STATUS_WAIT_TIMEOUT = 4u;
constexpr int EDGE_BATCH = 64;  // fan-out edges per batch of the adjoint: two records per lane
constexpr uint64_t WAIT_NS = 1000000000ull;  // bound of one wait for a warp's own copies (1 s)

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
// Rows r0..r3 (each one full tensor-map row) -> dst, dst + row, ... (dense).
__device__ __forceinline__ void gather4(void* dst, const CUtensorMap* map, int r0, int r1, int r2, int r3,
                                        uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
        "%4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void gather4_hint(void* dst, const CUtensorMap* map, int r0, int r1, int r2, int r3,
                                             uint64_t* bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes.L2::cache_hint [%0], "
        "[%1, {%2, %3, %4, %5, %6}], [%7], %8;" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(smem_u32(bar)),
        "l"(policy)
        : "memory");
}

// Tensor maps over the scratch rows of all tiles (act row = tile * n_act_rows + row in
// the tile, adj likewise with n_adj_rows).
struct RowMaps {
    const CUtensorMap* act;
    const CUtensorMap* adj;
    int arow0, grow0;  // this tile's first act / adj row
};

// Adjoint rows are re-read by the next few levels (as consumer adjoints): stored with
// an evict-last L2 policy (and discarded after their last reader).
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void st_row_hint(float* p, const VF& x, uint64_t pol) {
    static_assert(VEC == 4, "one 16-byte store per lane");
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(x.v[0]), "f"(x.v[1]),
                 "f"(x.v[2]), "f"(x.v[3]), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// Drop 128-byte lines from L2 without writing them back (their contents become
// undefined): used for adjoint rows whose last reader has run.
__device__ __forceinline__ void discard_l2_line(const void* p) {
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Per-warp staging state: NSLOT slots of slot_bytes<T>() and their mbarriers.
struct Stage {
    char* buf;
    uint64_t* bar;
    int* rows;            // [2][EDGE_BATCH]: the tensor-map rows of the current batch's two operands
    float4* coef;         // the batch's gate coefficients (forward, 32) or edge (c0, c1) pairs (EDGE_BATCH)
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
// Per warp: NSLOT slots, their mbarriers, and the batch's row table (2 x 32 int32,
// 16-byte aligned for int4 reads); the stride is rounded to 128 bytes so every slot (and
// every bulk-copy destination inside it) stays 16-byte aligned for every warp.
template <typename T>
__host__ __device__ constexpr int stage_rows_offset() {
    return (NSLOT * slot_bytes<T>() + NSLOT * 8 + 15) / 16 * 16;
}
template <typename T>
__host__ __device__ constexpr int warp_stage_bytes() {
    return (stage_rows_offset<T>() + 2 * EDGE_BATCH * 4 + 32 * 16 + 127) / 128 * 128;
}

template <typename T>
__device__ __forceinline__ Stage make_stage(char* smem, unsigned* status, const TileCtx& c) {
    Stage st;
    st.buf = smem + c.warp * warp_stage_bytes<T>();
    st.bar = reinterpret_cast<uint64_t*>(st.buf + NSLOT * slot_bytes<T>());
    st.rows = reinterpret_cast<int*>(st.buf + stage_rows_offset<T>());
    st.coef = reinterpret_cast<float4*>(st.buf + stage_rows_offset<T>() + 2 * EDGE_BATCH * 4);
    st.parity = 0;
    st.status = status;
    st.poisoned = false;
    return st;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for the phase of `bar` with the given parity: false after limit_ns
// nanoseconds (or 2^30 polls) without completion; the copies it counts are then given up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; it++) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 15) == 0 && (global_ns() - t0 > limit_ns || it > (1u << 30))) return false;
    }
}

// Warp-uniform: wait for the completion of slot s.  On expiry the warp records
// STATUS_WAIT_TIMEOUT and stops waiting for the rest of the launch.
__device__ __forceinline__ void stage_wait(Stage& st, int s) {
    if (!st.poisoned && !mbar_wait_bounded(st.bar + s, (st.parity >> s) & 1u, WAIT_NS)) {
        st.poisoned = true;
        if ((threadIdx.x & 31) == 0) atomicOr(st.status, STATUS_WAIT_TIMEOUT);
    }
    st.parity ^= 1u << s;
    __syncwarp();
}

// Diagnostic: one warp waits, with the step kernels' bounded wait, on an mbarrier
// whose phase nothing completes (expect_tx of one byte, no copy issued), and records
// the expiry in *status like the step kernels do.  No copy is in flight, so the
// kernel can return at once.
__global__ void bounded_wait_diag_kernel(unsigned* status, uint64_t limit_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (threadIdx.x == 0) mbar_expect_tx(&bar, 1u);  // the one arrival; one byte stays pending forever
    __syncwarp();
    if (!mbar_wait_bounded(&bar, 0u, limit_ns) && threadIdx.x == 0) atomicOr(status, STATUS_WAIT_TIMEOUT);
}

// Forward pass of one tile, input level: P = sigmoid(V) for the cone inputs (rows
// 0 .. n_cone_pi - 1 in every layout).
template <typename T>
__device__ void tile_inputs(const DevPlan& p, const float* __restrict__ V, int64_t ldv, T* act, const TileCtx& c) {
    for (int i0 = c.vw * UBATCH; i0 < p.n_cone_pi; i0 += c.nvw * UBATCH) {
        VF x[UBATCH];
#pragma unroll
        for (int u = 0; u < UBATCH; u++) {
            const int i = i0 + u;
            x[u] = vf_fill(0.0f);
            if (i < p.n_cone_pi) {
                const float* r = V + (int64_t)__ldg(&p.cone_pi_row[i]) * ldv + c.b;
#pragma unroll
                for (int q = 0; q < VEC; q++)
                    if (q < c.nvalid) x[u].v[q] = r[q];
            }
        }
#pragma unroll
        for (int u = 0; u < UBATCH; u++) {
            const int i = i0 + u;
            if (i < p.n_cone_pi) {
                VF y;
#pragma unroll
                for (int q = 0; q < VEC; q++) y.v[q] = sigmoidf_(x[u].v[q]);
                ActIO<T>::st(act + at(i, c), y);
            }
        }
    }
    fence_async_global();
    level_sync(c);
}

// Forward pass over cone levels l_lo .. l_hi (all of them, or with scratch_only the
// levels the layout does not keep: the re-evaluation of a segment).  Within a level each
// warp takes a contiguous run of gates; 32 gate records come in one coalesced load, and
// their input rows and coefficients go into the warp's row and coefficient tables in
// shared memory; the two input rows of each gate are gathered into shared memory (two
// gather4 loads per CHUNK = 4 gates, issued by lane 0 from the row table), NSLOT-1 chunks
// ahead of the computation.  gcoef: the 16 bilinear coefficient sets in shared memory.
template <typename T>
__device__ void forward_levels(const DevPlan& p, const DevAct& L, T* act, Stage& st, const float4* gcoef,
                               const RowMaps& rm, const TileCtx& c, int l_lo, int l_hi, bool scratch_only) {
    constexpr int ROWB = TILE * (int)sizeof(T);
    constexpr int SLOT = slot_bytes<T>();
    auto wanted = [&](int l) { return !scratch_only || __ldg(&L.stored[l]) == 0; };
    auto next_level = [&](int l) {
        do l++;
        while (l <= l_hi && !wanted(l));
        return l;
    };
    // This warp's gate run of level l, its first 32 gate records and the act row of the
    // level's first gate; those of the next level are loaded before the level barrier, so
    // that their latency overlaps the wait for the other warps.
    auto level_run = [&](int l, int& g0, int& g1, int& orow, int2& first) {
        const int lo = __ldg(&p.c_level_off[l]), hi = __ldg(&p.c_level_off[l + 1]);
        const int per = (hi - lo + c.nvw - 1) / c.nvw;
        g0 = lo + c.vw * per;
        g1 = min(g0 + per, hi);
        orow = __ldg(&L.act_off[l]) - lo;
        first = make_int2(0, 0);
        if (c.lane < g1 - g0) first = __ldg(&L.gate[g0 + c.lane - p.n_cone_pi]);
    };
    int g0 = 0, g1 = 0, orow = 0;
    int2 first = make_int2(0, 0);
    int l = l_lo;
    if (l <= l_hi && !wanted(l)) l = next_level(l);
    if (l <= l_hi) level_run(l, g0, g1, orow, first);
    while (l <= l_hi) {
        for (int base = g0; base < g1; base += 32) {
            const int cnt = min(32, g1 - base);
            int2 mine = first;
            if (base != g0) {
                mine = make_int2(0, 0);
                if (c.lane < cnt) mine = __ldg(&L.gate[base + c.lane - p.n_cone_pi]);
            }
            const int nch = (cnt + CHUNK - 1) / CHUNK;
            // per lane (= gate of the batch): tensor-map rows of both inputs, into the warp's
            // row table (lanes past cnt repeat the last gate, so a partial chunk does too), and
            // the gate code
            {
                const int x_row = rm.arow0 + (mine.x & 0x0FFFFFFF), y_row = rm.arow0 + mine.y;
                const int x_last = __shfl_sync(FULL, x_row, cnt - 1), y_last = __shfl_sync(FULL, y_row, cnt - 1);
                st.rows[c.lane] = c.lane < cnt ? x_row : x_last;
                st.rows[EDGE_BATCH + c.lane] = c.lane < cnt ? y_row : y_last;
                st.coef[c.lane] = gcoef[(uint32_t)mine.x >> 28];  // this lane's gate's (k0, k1, k2, k3)
                __syncwarp();
            }
            T* out = act + at(base + orow, c);
            auto issue = [&](int ch) {
                const int s = ch % NSLOT;
                // first inputs of the chunk's 4 gates -> rows 0..3, second inputs -> rows 4..7
                if (c.lane == 0) {
                    const int4 xr = *reinterpret_cast<const int4*>(st.rows + ch * CHUNK);
                    const int4 yr = *reinterpret_cast<const int4*>(st.rows + EDGE_BATCH + ch * CHUNK);
                    mbar_expect_tx(st.bar + s, (uint32_t)(2 * CHUNK * ROWB));
                    gather4(st.buf + s * SLOT, rm.act, xr.x, xr.y, xr.z, xr.w, st.bar + s);
                    gather4(st.buf + s * SLOT + CHUNK * ROWB, rm.act, yr.x, yr.y, yr.z, yr.w, st.bar + s);
                }
            };
            for (int ch = 0; ch < NSLOT - 1 && ch < nch; ch++) issue(ch);
            for (int ch = 0; ch < nch; ch++) {
                if (ch + NSLOT - 1 < nch) issue(ch + NSLOT - 1);
                const int s = ch % NSLOT;
                stage_wait(st, s);
                const char* sb = st.buf + s * SLOT;
                T* out_ch = out + ch * CHUNK * TILE;
                auto gate = [&](int j) {  // gate ch * CHUNK + j (< 32: at most 8 chunks of a batch)
                    const float4 k = st.coef[ch * CHUNK + j];
                    const VF x = ActIO<T>::ld(reinterpret_cast<const T*>(sb + j * ROWB) + c.lane * VEC);
                    const VF y = ActIO<T>::ld(reinterpret_cast<const T*>(sb + (CHUNK + j) * ROWB) + c.lane * VEC);
                    VF z;
                    // gate_apply on two samples per instruction (the same IEEE fma per element)
                    const float2 kw = make_float2(k.w, k.w), kz = make_float2(k.z, k.z);
                    const float2 ky = make_float2(k.y, k.y), kx = make_float2(k.x, k.x);
#pragma unroll
                    for (int q = 0; q < VEC; q += 2) {
                        const float2 a = make_float2(x.v[q], x.v[q + 1]), b = make_float2(y.v[q], y.v[q + 1]);
                        const float2 r = __ffma2_rn(__ffma2_rn(kw, a, kz), b, __ffma2_rn(ky, a, kx));
                        z.v[q] = r.x;
                        z.v[q + 1] = r.y;
                    }
                    ActIO<T>::st(out_ch + j * TILE, z);
                };
                if ((ch + 1) * CHUNK <= cnt) {  // a full chunk
#pragma unroll
                    for (int j = 0; j < CHUNK; j++) gate(j);
                } else {
#pragma unroll
                    for (int j = 0; j < CHUNK; j++)
                        if (ch * CHUNK + j < cnt) gate(j);
                }
                fence_async_shared();
                __syncwarp();
            }
        }
        l = next_level(l);
        if (l <= l_hi) level_run(l, g0, g1, orow, first);
        fence_async_global();
        level_sync(c);
    }
}

// inputs_ready: the previous step's update has written the inputs' act rows already.
template <typename T>
__device__ void tile_forward(const DevPlan& p, const DevAct& L, const float* __restrict__ V, int64_t ldv, T* act,
                             Stage& st, const float4* gcoef, const RowMaps& rm, const TileCtx& c,
                             bool inputs_ready = false) {
    if (!inputs_ready) tile_inputs<T>(p, V, ldv, act, c);
    forward_levels<T>(p, L, act, st, gcoef, rm, c, 1, p.n_clev, false);
}

// Per-sample loss sum_j (Y_j - T_j)^2, FP32, fixed order (warp-strided partials, then warp order).
template <typename T>
__device__ void tile_loss(const DevPlan& p, const DevAct& L, const T* act, float* loss, const TileCtx& c) {
    __shared__ VF part[step_threads<T>() / 32][32];
    VF acc = vf_fill(0.0f);
    for (int j = c.warp; j < p.n_out; j += c.nw) {
        const VF y = ActIO<T>::ldcg(act + at(__ldg(&L.out_row[j]), c));
        const float t = p.out_target[j];
#pragma unroll
        for (int q = 0; q < VEC; q++) acc.v[q] = fmaf(y.v[q] - t, y.v[q] - t, acc.v[q]);
    }
    part[c.warp][c.lane] = acc;
    __syncthreads();
    if (c.warp == 0) {
        VF sum = vf_fill(0.0f);
        for (int w = 0; w < c.nw; w++)
#pragma unroll
            for (int q = 0; q < VEC; q++) sum.v[q] += part[w][c.lane].v[q];
#pragma unroll
        for (int q = 0; q < VEC; q++)
            if (q < c.nvalid) loss[c.b + q] = sum.v[q];
    }
    __syncthreads();
}

// Adjoints of cone nodes [lo, hi) (gather form of Eq. 8): each warp takes a
// contiguous run of nodes, whose fan-out edges are contiguous in the CSR and
// are summed in CSR order.  An edge contributes ga * (c0 + c1 * A_sibling)
// with ga the consumer's adjoint row, or for an output seed the seed row (the
// per-sample weight of the loss, written at the start of the backward pass).  Up to 64
// edge records (two per lane) fill the warp's row and coefficient tables; the
// consumer-adjoint and sibling rows are gathered into shared memory (one gather4 load
// each per CHUNK = 4 edges).
// This warp's node run [u0, u1) of a cone level with the CSR offsets of its first
// 31 nodes and its first 32 fan-out edges, loaded ahead (before the barrier of
// the level above) so that the three dependent loads do not stall the level.
struct AdjRun {
    int u0, u1, off;
    int arow;  // adj row of node u0
    int4 first;
};
__device__ __forceinline__ AdjRun adj_run(const DevPlan& p, const DevAct& L, int l, const TileCtx& c) {
    const int lo = l == 0 ? 0 : __ldg(&p.c_level_off[l]);
    const int hi = l == 0 ? p.n_cone_pi : __ldg(&p.c_level_off[l + 1]);
    AdjRun r;
    int set = -1;
#pragma unroll
    for (int k = 0; k < DevPlan::ADJ_RUN_SETS; k++)
        if (p.adj_run_w[k] == c.nvw) set = k;
    if (p.adj_run != nullptr && set >= 0) {  // runs of about equal fan-out edge counts
        const int32_t* t = p.adj_run + p.adj_run_base[set] + (int64_t)l * (c.nvw + 1) + c.vw;
        r.u0 = __ldg(t);
        r.u1 = __ldg(t + 1);
    } else {  // equal node counts
        const int per = (hi - lo + c.nvw - 1) / c.nvw;
        r.u0 = min(lo + c.vw * per, hi);
        r.u1 = min(r.u0 + per, hi);
    }
    r.arow = (int)((l == 0 ? (int64_t)lo : adj_level_row(p, l, lo)) + (r.u0 - lo));
    r.off = 0;
    r.first = make_int4(-1, 0, 0, 0);
    if (r.u0 < r.u1) {
        const int nn = min(31, r.u1 - r.u0);
        r.off = (c.lane <= nn) ? __ldg(&p.fo_off[r.u0 + c.lane]) : 0;
        const int e_begin = __shfl_sync(FULL, r.off, 0), e_end = __shfl_sync(FULL, r.off, nn);
        if (c.lane < min(32, e_end - e_begin)) r.first = __ldg(&L.edge[e_begin + c.lane]);
    }
    return r;
}

template <typename T>
__device__ void level_adjoint(const DevPlan& p, const DevAct& L, const AdjRun& run, const T* act, float* adj,
                              Stage& st, const RowMaps& rm, const TileCtx& c) {
    constexpr int ROWB = TILE * (int)sizeof(T);
    constexpr int ROWF = TILE * 4;
    constexpr int SLOT = slot_bytes<T>();
    const uint64_t stream_policy = policy_evict_first();
    const uint64_t keep_policy = policy_evict_last();
    const int u0 = run.u0, u1 = run.u1;
    for (int ua = u0; ua < u1; ua += 31) {
        const int nn = min(31, u1 - ua);
        const int off = ua == u0 ? run.off : ((c.lane <= nn) ? __ldg(&p.fo_off[ua + c.lane]) : 0);
        const int e_begin = __shfl_sync(FULL, off, 0), e_end = __shfl_sync(FULL, off, nn);
        int k = 0;                         // nodes of this run stored so far
        float* node_row = adj + at(run.arow + (ua - u0), c);  // where the next node's adjoint goes
        VF acc = vf_fill(0.0f);
        for (int base = e_begin; base < e_end; base += EDGE_BATCH) {
            // up to 64 edges: edge base + lane in `mine`, base + 32 + lane in `mine2`
            const int cnt = min(EDGE_BATCH, e_end - base);
            int4 mine = run.first, mine2 = make_int4(-1, 0, 0, 0);
            if (ua != u0 || base != e_begin) {
                mine = make_int4(-1, 0, 0, 0);
                if (c.lane < cnt) mine = __ldg(&L.edge[base + c.lane]);
            }
            if (32 + c.lane < cnt) mine2 = __ldg(&L.edge[base + 32 + c.lane]);
            const int nch = (cnt + CHUNK - 1) / CHUNK;
            // per edge: tensor-map rows of the consumer adjoint (the seed row for an output seed)
            // and of the sibling, into the warp's row table (entries past cnt repeat the last
            // edge, so a partial chunk does too), and the partial's (c0, c1)
            {
                const int g_row = rm.grow0 + max(mine.x, 0), s_row = rm.arow0 + (mine.y & 0x7FFFFFFF);
                const int g_row2 = rm.grow0 + max(mine2.x, 0), s_row2 = rm.arow0 + (mine2.y & 0x7FFFFFFF);
                const bool last_lo = cnt <= 32;  // the batch's last edge is in `mine`
                const int g_last = __shfl_sync(FULL, last_lo ? g_row : g_row2, (cnt - 1) & 31);
                const int s_last = __shfl_sync(FULL, last_lo ? s_row : s_row2, (cnt - 1) & 31);
                st.rows[c.lane] = c.lane < cnt ? g_row : g_last;
                st.rows[32 + c.lane] = 32 + c.lane < cnt ? g_row2 : g_last;
                st.rows[EDGE_BATCH + c.lane] = c.lane < cnt ? s_row : s_last;
                st.rows[EDGE_BATCH + 32 + c.lane] = 32 + c.lane < cnt ? s_row2 : s_last;
                float2* cc = reinterpret_cast<float2*>(st.coef);
                cc[c.lane] = make_float2(__int_as_float(mine.z), __int_as_float(mine.w));
                cc[32 + c.lane] = make_float2(__int_as_float(mine2.z), __int_as_float(mine2.w));
                __syncwarp();
            }
            // edges that close their node's sum (the node's adjoint row is stored there)
            const unsigned last_lo = __ballot_sync(FULL, c.lane < cnt && mine.y < 0);
            const unsigned last_hi = __ballot_sync(FULL, 32 + c.lane < cnt && mine2.y < 0);
            auto issue = [&](int ch) {
                const int s = ch % NSLOT;
                // consumer adjoints -> the 4 fp32 rows, siblings -> the 4 act rows
                if (c.lane == 0) {
                    const int4 gr = *reinterpret_cast<const int4*>(st.rows + ch * CHUNK);
                    const int4 sr = *reinterpret_cast<const int4*>(st.rows + EDGE_BATCH + ch * CHUNK);
                    char* sb = st.buf + s * SLOT;
                    mbar_expect_tx(st.bar + s, (uint32_t)(CHUNK * ROWF + CHUNK * ROWB));
                    gather4(sb, rm.adj, gr.x, gr.y, gr.z, gr.w, st.bar + s);
                    gather4_hint(sb + CHUNK * ROWF, rm.act, sr.x, sr.y, sr.z, sr.w, st.bar + s, stream_policy);
                }
            };
            for (int ch = 0; ch < NSLOT - 1 && ch < nch; ch++) issue(ch);
            for (int ch = 0; ch < nch; ch++) {
                if (ch + NSLOT - 1 < nch) issue(ch + NSLOT - 1);
                const int s = ch % NSLOT;
                stage_wait(st, s);
                const char* sb = st.buf + s * SLOT;
                // bit j: edge ch * CHUNK + j closes its node (CHUNK divides 32)
                const unsigned chunk_last = ch * CHUNK < 32 ? last_lo >> (ch * CHUNK) : last_hi >> (ch * CHUNK - 32);
                auto edge = [&](int j) {  // edge ch * CHUNK + j (< 64: at most 16 chunks of a batch)
                    const float2 cc = reinterpret_cast<const float2*>(st.coef)[ch * CHUNK + j];
                    const VF ga = ActIO<float>::ld(reinterpret_cast<const float*>(sb + j * ROWF) + c.lane * VEC);
                    const VF sv = ActIO<T>::ld(reinterpret_cast<const T*>(sb + CHUNK * ROWF + j * ROWB) + c.lane * VEC);
                    const float2 c1 = make_float2(cc.y, cc.y), c0 = make_float2(cc.x, cc.x);
#pragma unroll
                    for (int q = 0; q < VEC; q += 2) {
                        const float2 d = __ffma2_rn(c1, make_float2(sv.v[q], sv.v[q + 1]), c0);
                        const float2 r = __ffma2_rn(make_float2(ga.v[q], ga.v[q + 1]), d,
                                                    make_float2(acc.v[q], acc.v[q + 1]));
                        acc.v[q] = r.x;
                        acc.v[q + 1] = r.y;
                    }
                    if ((chunk_last >> j) & 1u) {
                        st_row_hint(node_row, acc, keep_policy);
                        node_row += TILE;
                        acc = vf_fill(0.0f);
                        k++;
                    }
                };
                if ((ch + 1) * CHUNK <= cnt) {  // a full chunk
#pragma unroll
                    for (int j = 0; j < CHUNK; j++) edge(j);
                } else {
#pragma unroll
                    for (int j = 0; j < CHUNK; j++)
                        if (ch * CHUNK + j < cnt) edge(j);
                }
                fence_async_shared();
                __syncwarp();
            }
        }
        while (k < nn) {  // (none left: every node's range ends with a marked edge)
            ActIO<float>::st(node_row, acc);
            node_row += TILE;
            acc = vf_fill(0.0f);
            k++;
        }
    }
}


// Discard, from L2, this tile's adjoint rows of cone level l (level 0 = the
// inputs); the whole CTA shares the 128-byte lines.
__device__ __forceinline__ void discard_adj_rows(const DevPlan& p, int l, const float* adj, const TileCtx& c) {
    const int lo = l == 0 ? 0 : __ldg(&p.c_level_off[l]);
    const int hi = l == 0 ? p.n_cone_pi : __ldg(&p.c_level_off[l + 1]);
    const int64_t row = l == 0 ? 0 : adj_level_row(p, l, lo);
    const char* b = reinterpret_cast<const char*>(adj);
    constexpr int LINES_PER_ROW = TILE * 4 / 128;
    const int n = (hi - lo) * LINES_PER_ROW;
    const int stride = (c.split ? 2 : 1) * (int)blockDim.x;
    for (int i = c.rank * (int)blockDim.x + (int)threadIdx.x; i < n; i += stride)
        discard_l2_line(b + (size_t)row * TILE * 4 + (size_t)i * 128);
}

// Discard, from L2, the ring rows whose last reader was level l (their dirty lines are
// then never written back); the whole CTA (both CTAs of a split tile) shares the lines.
__device__ __forceinline__ void discard_dead_rows(const DevPlan& p, int l, const float* adj, const TileCtx& c) {
    const int lo = __ldg(&p.dead_off[l]), hi = __ldg(&p.dead_off[l + 1]);
    const char* b = reinterpret_cast<const char*>(adj);
    constexpr int LINES_PER_ROW = TILE * 4 / 128;
    const int n = (hi - lo) * LINES_PER_ROW;
    const int stride = (c.split ? 2 : 1) * (int)blockDim.x;
    for (int i = c.rank * (int)blockDim.x + (int)threadIdx.x; i < n; i += stride) {
        const int row = __ldg(&p.dead_row[lo + i / LINES_PER_ROW]);
        discard_l2_line(b + (size_t)row * TILE * 4 + (size_t)(i % LINES_PER_ROW) * 128);
    }
}

// Discard the whole adjoint scratch of this tile (after the input level has been read).
__device__ __forceinline__ void discard_adj_all(const DevPlan& p, const float* adj, const TileCtx& c) {
    const char* b = reinterpret_cast<const char*>(adj);
    constexpr int LINES_PER_ROW = TILE * 4 / 128;
    const int64_t n = p.n_adj_rows * LINES_PER_ROW;
    const int stride = (c.split ? 2 : 1) * (int)blockDim.x;
    for (int64_t i = c.rank * (int)blockDim.x + (int)threadIdx.x; i < n; i += stride)
        discard_l2_line(b + (size_t)i * 128);
}

// Backward pass of one tile over levels n_clev..0.  Under a recomputation layout
// (L.k > 0) each segment's unkept levels are evaluated again, from the kept levels
// below it, before its adjoints; the forward pass leaves the top two segments'
// scratch valid (buffers J % 2 and (J - 1) % 2), so those are not re-evaluated.  The
// input level's adjoints (of P) are turned into dL/dV and either stored (gV) or
// applied by the optimiser, UBATCH rows at a time.
template <typename T, bool UPDATE>
__device__ void tile_backward(const DevPlan& p, const DevAct& L, const OptParams& o, float* V, float* m, float* v,
                              float* gV, int64_t ldv, T* act, float* adj, const float* grad_loss,
                              const AdamCorr& ac, Stage& st, const float4* gcoef, const RowMaps& rm,
                              const TileCtx& c, bool next_inputs = false) {
    // the seed row: each sample's weight of its loss (1, or grad_loss), read by the seed edges
    if (c.warp == 0 && c.rank == 0) {
        VF seed_scale = vf_fill(1.0f);
        if (grad_loss != nullptr)
#pragma unroll
            for (int q = 0; q < VEC; q++) seed_scale.v[q] = q < c.nvalid ? grad_loss[c.b + q] : 0.0f;
        ActIO<float>::st(adj + at(p.seed_row, c), seed_scale);
    }
    fence_async_global();
    level_sync(c);
    const int top_seg = L.k > 0 && p.n_clev > 0 ? (p.n_clev - 1) / L.k : 0;
    AdjRun run = adj_run(p, L, p.n_clev, c);
    for (int l = p.n_clev; l >= 0; l--) {
        if (L.k > 0 && l >= 1 && (l % L.k == 0 || l == p.n_clev)) {  // l: the top level of its segment
            const int j = (l - 1) / L.k;
            if (j + 2 <= top_seg) forward_levels<T>(p, L, act, st, gcoef, rm, c, j * L.k + 1, l, true);
        }
        level_adjoint<T>(p, L, run, act, adj, st, rm, c);
        if (l > 0) run = adj_run(p, L, l - 1, c);
        fence_async_global();
        level_sync(c);
        // Adjoint rows of level l + span have no reader below level l.  (In the ring, their
        // slot is level l - 1's, written right after this barrier: a discard there would
        // race with those stores, so ring slots are only discarded at the end.)
        if (p.adj_slots == 0 && l + p.max_span <= p.n_clev) discard_adj_rows(p, l + p.max_span, adj, c);
        if (p.adj_slots > 0 && p.dead_off) discard_dead_rows(p, l, adj, c);
    }
    // The input level's adjoints become dL/dV and the update; with next_inputs the update
    // also writes P = sigmoid(V) of the new logits into the inputs' act rows, where the next
    // step's forward pass starts (after the barrier above: until then the level-0 edges may
    // still gather those rows as siblings).
    const bool adam = UPDATE && o.opt == 0;
    for (int i0 = c.vw * UBATCH; i0 < p.n_cone_pi; i0 += c.nvw * UBATCH) {
        VF vv[UBATCH], pb[UBATCH], mm[UBATCH], ss[UBATCH];
        int64_t r[UBATCH];
#pragma unroll
        for (int u = 0; u < UBATCH; u++) {
            const int i = i0 + u;
            r[u] = 0;
            vv[u] = mm[u] = ss[u] = pb[u] = vf_fill(0.0f);
            if (i < p.n_cone_pi) {
                r[u] = (int64_t)__ldg(&p.cone_pi_row[i]) * ldv + c.b;
                pb[u] = ActIO<float>::ldcg(adj + at(i, c));  // possibly written by the other CTA
#pragma unroll
                for (int q = 0; q < VEC; q++) {
                    if (q < c.nvalid) {
                        vv[u].v[q] = V[r[u] + q];
                        if (adam) {
                            mm[u].v[q] = m[r[u] + q];
                            ss[u].v[q] = v[r[u] + q];
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < UBATCH; u++) {
            if (i0 + u >= p.n_cone_pi) continue;
            VF y;
#pragma unroll
            for (int q = 0; q < VEC; q++) {
                float nv = 0.0f;  // samples past B: sigmoid(0), as the input pass writes them
                if (q < c.nvalid)
                    nv = input_update<UPDATE>(o, V, m, v, gV, r[u] + q, vv[u].v[q], pb[u].v[q], mm[u].v[q],
                                              ss[u].v[q], ac.step[q], ac.bc2s[q]);
                y.v[q] = sigmoidf_(nv);
            }
            if (next_inputs) ActIO<T>::st(act + at(i0 + u, c), y);
        }
    }
    fence_async_global();  // the inputs' act rows are gathered by the next forward pass
    level_sync(c);
    if (p.adj_slots == 0)
        for (int l = 0; l < p.max_span && l <= p.n_clev; l++) discard_adj_rows(p, l, adj, c);
    else
        discard_adj_all(p, adj, c);
}

// Scratch of tile t: act rows [n_act_rows][TILE] from element t * n_act_rows * TILE, adj
// rows [n_adj_rows][TILE] from element t * n_adj_rows * TILE.
// Dynamic shared memory: warp_stage_bytes<T>() per warp (slots + mbarriers).
template <typename T>
__device__ __forceinline__ Stage init_stage(char* smem, const DevPlan& p, float4* gcoef, const TileCtx& c) {
    Stage st = make_stage<T>(smem, p.status, c);
    if (c.lane == 0)
        for (int s = 0; s < NSLOT; s++) mbar_init(st.bar + s, 1);
    if (threadIdx.x < 16) gcoef[threadIdx.x] = gate_coeffs(threadIdx.x);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();
    return st;
}

template <typename T>
__global__ void __launch_bounds__(step_threads<T>(), 1) forward_kernel(DevPlan p, const float* V, int64_t ldv, T* act,
                                                                  float* loss, int64_t B,
                                                                  const __grid_constant__ CUtensorMap amap) {
    extern __shared__ __align__(128) char smem[];
    __shared__ float4 gcoef[16];
    const TileCtx c = tile_ctx(B);
    Stage st = init_stage<T>(smem, p, gcoef, c);
    T* a = act + (size_t)c.tile * (size_t)p.full.n_act_rows * TILE;
    const RowMaps rm{&amap, &amap, (int)(c.tile * p.full.n_act_rows), 0};
    tile_forward<T>(p, p.full, V, ldv, a, st, gcoef, rm, c);
    if (loss) tile_loss<T>(p, p.full, a, loss, c);
}

template <typename T>
__global__ void __launch_bounds__(step_threads<T>(), 1) backward_kernel(DevPlan p, const float* V, int64_t ldv,
                                                                   const T* act, float* adj, const float* grad_loss,
                                                                   float* gV, int64_t B,
                                                                   const __grid_constant__ CUtensorMap amap,
                                                                   const __grid_constant__ CUtensorMap gmap) {
    extern __shared__ __align__(128) char smem[];
    __shared__ float4 gcoef[16];
    const TileCtx c = tile_ctx(B);
    Stage st = init_stage<T>(smem, p, gcoef, c);
    OptParams o;
    AdamCorr ac;
#pragma unroll
    for (int q = 0; q < VEC; q++) ac.step[q] = ac.bc2s[q] = 1.0f;
    const RowMaps rm{&amap, &gmap, (int)(c.tile * p.full.n_act_rows), (int)(c.tile * p.n_adj_rows)};
    tile_backward<T, false>(p, p.full, o, const_cast<float*>(V), nullptr, nullptr, gV, ldv,
                            const_cast<T*>(act) + (size_t)c.tile * (size_t)p.full.n_act_rows * TILE,
                            adj + (size_t)c.tile * (size_t)p.n_adj_rows * TILE, grad_loss, ac, st, gcoef, rm, c);
}

// The fused hot loop: n_steps x (forward, loss, adjoint, update) for one tile,
// at Adam steps t0 + s (+ age[b] per sample when age is given).
// SPLIT: launched in clusters of two CTAs per tile (tiles tile0, tile0 + 1, ...).
template <typename T, bool SPLIT>
__global__ void __launch_bounds__(step_threads<T>(), 1) steps_kernel(DevPlan p, DevAct L, OptParams o, float* V, float* m,
                                                                float* v, int64_t ldv, T* act, float* adj, float* loss,
                                                                int t0, const int32_t* age, int n_steps, int64_t B,
                                                                int tile0, const __grid_constant__ CUtensorMap amap,
                                                                const __grid_constant__ CUtensorMap gmap) {
    extern __shared__ __align__(128) char smem[];
    __shared__ float4 gcoef[16];
    const TileCtx c = tile_ctx(B, tile0, SPLIT);
    Stage st = init_stage<T>(smem, p, gcoef, c);
    T* a = act + (size_t)c.tile * (size_t)L.n_act_rows * TILE;
    float* g = adj + (size_t)c.tile * (size_t)p.n_adj_rows * TILE;
    const RowMaps rm{&amap, &gmap, (int)(c.tile * L.n_act_rows), (int)(c.tile * p.n_adj_rows)};
#pragma unroll 1
    for (int s = 0; s < n_steps; s++) {
        AdamCorr ac;
        if (o.opt == 0) ac = adam_corr(o, age, t0 + s, c);
        tile_forward<T>(p, L, V, ldv, a, st, gcoef, rm, c, s > 0);
        if (loss && s == n_steps - 1 && c.rank == 0) tile_loss<T>(p, L, a, loss, c);
        tile_backward<T, true>(p, L, o, V, m, v, nullptr, ldv, a, g, nullptr, ac, st, gcoef, rm, c,
                               s + 1 < n_steps);
    }
}

template <typename T>
constexpr size_t stage_smem() {
    return (size_t)(step_threads<T>() / 32) * warp_stage_bytes<T>();
}

// Opt the step kernels into the dynamic shared memory they use (once per type and device).
template <typename T>
cudaError_t prepare_tile_kernels() {
    static PerDeviceOnce once;
    return once.run([] {
        const int bytes = (int)stage_smem<T>();
        cudaError_t e = cudaFuncSetAttribute(forward_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(backward_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(steps_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(steps_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        return e;
    });
}

__global__ void opt_update_kernel(DevPlan p, OptParams o, float* V, float* m, float* v, const float* gV, int64_t ldv,
                                  int t, int64_t B) {
    const int64_t n = (int64_t)p.n_cone_pi * B;
    float step_size = 0.0f, bc2s = 1.0f;
    if (o.opt == 0) adam_bias(o, t, step_size, bc2s);
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

template <typename T>
constexpr CUtensorMapDataType tmap_type() {
    return sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                          : (std::is_same<T, __half>::value ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                            : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
}

// Maps over the act (type T, layout L) and adj (fp32) scratch of `tiles` tiles: one row
// per (tile, scratch row), TILE elements wide, box = one row (for tile::gather4).
// With an empty cone the maps stay zero and unused.
template <typename T>
cudaError_t row_maps(const DevPlan& p, const DevAct& L, const void* act, const float* adj, unsigned tiles,
                     CUtensorMap* amap, CUtensorMap* gmap) {
    memset(amap, 0, sizeof(*amap));
    memset(gmap, 0, sizeof(*gmap));
    if (p.n_cone == 0 || tiles == 0) return cudaSuccess;
    const int64_t arows = (int64_t)tiles * L.n_act_rows, grows = (int64_t)tiles * p.n_adj_rows;
    if (arows > 0x7fffffff || grows > 0x7fffffff) return cudaErrorInvalidValue;  // row coordinates are int32
    if (act && !encode_2d(amap, act, tmap_type<T>(), (int)sizeof(T), arows, TILE, TILE, TILE, 1,
                          CU_TENSOR_MAP_SWIZZLE_NONE))
        return cudaErrorInvalidValue;
    if (adj && !encode_2d(gmap, adj, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, grows, TILE, TILE, TILE, 1,
                          CU_TENSOR_MAP_SWIZZLE_NONE))
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

template <typename T>
cudaError_t forward_launch(const DevPlan& p, const float* V, int64_t ldv, void* act, float* loss, int64_t B,
                           cudaStream_t s) {
    cudaError_t e = prepare_tile_kernels<T>();
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((B + TILE - 1) / TILE);
    CUtensorMap amap, gmap;
    if ((e = row_maps<T>(p, p.full, act, nullptr, grid, &amap, &gmap)) != cudaSuccess) return e;
    forward_kernel<T><<<grid, step_threads<T>(), stage_smem<T>(), s>>>(p, V, ldv, (T*)act, loss, B, amap);
    return cudaGetLastError();
}

template <typename T>
cudaError_t backward_launch(const DevPlan& p, const float* V, int64_t ldv, const void* act, float* adj,
                            const float* grad_loss, float* gV, int64_t B, cudaStream_t s) {
    cudaError_t e = prepare_tile_kernels<T>();
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((B + TILE - 1) / TILE);
    CUtensorMap amap, gmap;
    if ((e = row_maps<T>(p, p.full, act, adj, grid, &amap, &gmap)) != cudaSuccess) return e;
    backward_kernel<T><<<grid, step_threads<T>(), stage_smem<T>(), s>>>(p, V, ldv, (const T*)act, adj, grad_loss, gV, B,
                                                                   amap, gmap);
    return cudaGetLastError();
}

template <typename T>
cudaError_t steps_launch(const DevPlan& p, const DevAct& L, const OptParams& o, float* V, float* m, float* v,
                         int64_t ldv, void* act, float* adj, float* loss, int t0, const int32_t* age, int n_steps,
                         int64_t B, cudaStream_t s) {
    cudaError_t e = prepare_tile_kernels<T>();
    if (e != cudaSuccess) return e;
    const int tiles = (int)((B + TILE - 1) / TILE);
    CUtensorMap amap, gmap;
    if ((e = row_maps<T>(p, L, act, adj, (unsigned)tiles, &amap, &gmap)) != cudaSuccess) return e;
    // Whole waves of tiles run one CTA per tile; a last, partial wave of at most half
    // the SMs runs in split mode (two CTAs of a cluster per tile) so that it fills them.
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
        return cudaErrorInvalidDevice;
    int main_tiles = tiles - tiles % sms;
    if (2 * (tiles - main_tiles) > sms) main_tiles = tiles;
    const int tail = tiles - main_tiles;
    if (main_tiles > 0) {
        steps_kernel<T, false><<<(unsigned)main_tiles, step_threads<T>(), stage_smem<T>(), s>>>(
            p, L, o, V, m, v, ldv, (T*)act, adj, loss, t0, age, n_steps, B, 0, amap, gmap);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (tail > 0) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(2 * tail), 1, 1);
        cfg.blockDim = dim3(step_threads<T>(), 1, 1);
        cfg.dynamicSmemBytes = stage_smem<T>();
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, steps_kernel<T, true>, p, L, o, V, m, v, ldv, (T*)act, adj, loss, t0, age,
                               n_steps, B, main_tiles, amap, gmap);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace

void step_warp_counts(int32_t out[DevPlan::ADJ_RUN_SETS]) {
    out[0] = step_threads<float>() / 32;
    out[1] = 2 * out[0];
    out[2] = step_threads<__half>() / 32;
    out[3] = 2 * out[2];
}

// ------------------------------------------------------------ launchers --
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

cudaError_t launch_steps(const DevPlan& p, const DevAct& L, int act_type, const OptParams& o, float* V, float* m,
                         float* v, int64_t ldv, void* act, float* adj, float* loss, int t0, int n_steps, int64_t B,
                         cudaStream_t s, const int32_t* age) {
    if (B == 0 || n_steps <= 0) return cudaSuccess;
    if (steps_use_resident(p, act_type))
        return launch_steps_resident(p, act_type, o, V, m, v, ldv, loss, t0, n_steps, B, s, age);
    if (p.step_kernel == STEP_KERNEL_RESIDENT) return cudaErrorInvalidValue;
    switch (act_type) {
    case ACT_F32: return steps_launch<float>(p, L, o, V, m, v, ldv, act, adj, loss, t0, age, n_steps, B, s);
    case ACT_BF16: return steps_launch<__nv_bfloat16>(p, L, o, V, m, v, ldv, act, adj, loss, t0, age, n_steps, B, s);
    default: return steps_launch<__half>(p, L, o, V, m, v, ldv, act, adj, loss, t0, age, n_steps, B, s);
    }
}

cudaError_t launch_bounded_wait_diag(unsigned* status, uint64_t limit_ns, cudaStream_t s) {
    bounded_wait_diag_kernel<<<1, 32, 0, s>>>(status, limit_ns);
    return cudaGetLastError();
}

cudaError_t launch_opt_update(const DevPlan& p, const OptParams& o, float* V, float* m, float* v, const float* gV,
                              int64_t ldv, int t, int64_t B, cudaStream_t s) {
    const int64_t n = (int64_t)p.n_cone_pi * B;
    if (n == 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 148 * 32);
    opt_update_kernel<<<grid, 256, 0, s>>>(p, o, V, m, v, gV, ldv, t, B);
    return cudaGetLastError();
}

}  // namespace sat
