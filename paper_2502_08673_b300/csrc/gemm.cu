// Dense BF16 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a) with a
// fused epilogue, for the proposal network's layers.
//
//   D[m][n] = sum_k A[m][k] * B[n][k]      (A: [M][lda], B: [N][ldb], both K-major bf16)
//   out = epi(D + bias[n])                 (epi: identity / GELU / times GELU'(Z[m][n]))
//
// Persistent and warp-specialised: one CTA per SM walks 128 x BN output tiles
// (BN = 64, 128 or 256).
//   warp 0      TMA producer: cp.async.bulk.tensor loads of 64-deep K chunks of
//               A and B into a ring of shared-memory stages;
//   warp 1      MMA issuer: one thread issues tcgen05.mma (M = 128, N = BN,
//               K = 16) per K slice into a TMEM accumulator, and commits each
//               stage back to the producer;
//   warps 2..17 epilogue: tcgen05.ld of the finished accumulator, bias /
//               activation / scale, then each 128 x 16 chunk is staged in
//               shared memory and written by a TMA tensor store (16-byte
//               direct stores where an output is not 16-byte aligned).
// Two TMEM accumulators alternate between tiles, so the epilogue of tile i
// runs while the MMAs of tile i+1 execute.  Operands sit in shared memory in
// the 128-byte-swizzled K-major layout that one TMA box of 64 K-elements x rows
// writes (each row's 128 bytes in 16-byte granules permuted by row mod 8, 8-row
// groups 1 KB apart); the 16-deep K slices of a chunk start 32 bytes apart
// inside that swizzle atom.  Out-of-range rows and K columns are zero-filled by
// TMA.
// Every mbarrier wait is bounded in time; an expired wait sets bit 3 of the
// status word and every role of the CTA stops, after letting its own copies
// and MMAs in flight finish.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "device.hpp"
#include "gemm.hpp"
#include "tmap.hpp"

namespace sat {
namespace {

constexpr int BM = 128;
constexpr int BK = 64;                               // K elements per stage: one 128-byte swizzle row
constexpr int EPI_GROUPS = 4;                        // column groups of the epilogue, 4 warps (128 rows) each
constexpr int N_EPI_WARPS = 4 * EPI_GROUPS;
constexpr int W = 16;                                // columns per epilogue chunk
constexpr int GEMM_THREADS = 64 + 32 * N_EPI_WARPS;  // + producer warp + MMA warp
constexpr uint64_t WAIT_NS = 2000000000ull;          // bound of one mbarrier wait (2 s)

template <int BN>
struct Cfg {
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;  // a multiple of 1024
    static constexpr int STAGES = BN == 256 ? 3 : (BN == 128 ? 4 : 6);
    static constexpr int RING = STAGES * STAGE;
    static constexpr int STAGING = EPI_GROUPS * 2 * 128 * W * 4;  // two FP32 chunk buffers per column group
    // barriers: full[STAGES], empty[STAGES], tmem_full[2], tmem_empty[2], done
    static constexpr int N_BAR = 2 * STAGES + 5;
    static constexpr int SMEM = 1024 + RING + STAGING + 8 * N_BAR + 16;  // + slack to align the ring to 1 KB
    static constexpr int TMEM_COLS = 2 * BN;
};

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the completion of the phase of parity `parity`.  Returns false when
// the CTA's abort flag is (or becomes) set, or after WAIT_NS, when it sets the
// flag and bit 3 of the status word itself.  With honour_abort = false the wait
// ignores the flag (used to drain copies and MMAs in flight before exit).
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile uint32_t* abort, unsigned* status,
                          bool honour_abort = true) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; it++) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 63) == 0) {
            if (honour_abort && *abort) return false;
            if (global_ns() - t0 > WAIT_NS || it > (1u << 30)) {
                *abort = 1u;
                atomicOr(status, 8u);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// Shared-memory matrix descriptor, K-major with 128-byte swizzle: start address,
// leading offset 16 B (unused when one MMA's K extent lies inside the swizzle
// row), stride between 8-row groups 1024 B, descriptor version 1, layout type 2
// (128-byte swizzle).  The tile base must be 1 KB aligned (base offset 0).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)2u << 61;
    return d;
}

// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, N, M = 128.
__host__ __device__ constexpr uint32_t instr_desc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ float gelu_exact(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

struct Flags {
    bool vec_f32, vec_bf16, vec_pre;                       // direct stores: 16-byte accesses allowed
    bool tma_pre, tma_f32, tma_bf16, tma_tbf16, tma_tf32;  // staged TMA stores available
};

// Store tensor maps of the outputs that take the staged path.
struct StoreMaps {
    CUtensorMap pre, f32, bf16, tbf16, tf32;
};

// Staged epilogue: a 128-row x W-column chunk is written to a shared-memory
// buffer in the layout of the output's TMA box, then stored by one thread with
// cp.async.bulk.tensor.  Each column group of the epilogue warps (4 warps: 128
// threads, all 128 rows) owns two such buffers and alternates between them.
enum OutKind { OUT_R32 = 0, OUT_R16 = 1, OUT_T32 = 2, OUT_T16 = 3 };
constexpr int STG_BYTES = 128 * W * 4;

struct Stager {
    uint32_t base;  // two buffers of STG_BYTES, 1 KB aligned
    int buf;
    int bar_id;     // named barrier of the column group
    bool issuer;    // the thread that issues the group's TMA stores
};

__device__ __forceinline__ void named_sync(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }

__device__ __forceinline__ void st_shared_v4(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(x), "r"(y), "r"(z), "r"(w) : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// Row r (0..127) of the chunk holds x[0..15].  Layouts of the buffer, matching the boxes:
//   OUT_R32  [128 rows][16 f32]   rows of 64 B, 16-byte granule k of row r at k ^ ((r / 2) mod 4)  (64-byte swizzle)
//   OUT_R16  [128 rows][16 bf16]  rows of 32 B, granule k of row r at k ^ ((r / 4) mod 2)        (32-byte swizzle)
//   OUT_T32  [16 cols][128 f32]   transposed, no swizzle
//   OUT_T16  [16 cols][128 bf16]  transposed, no swizzle
// Every thread of the group executes this (it contains two named barriers);
// `live` = false skips only the store itself.
template <int KIND>
__device__ __forceinline__ void staged_store(Stager& s, const CUtensorMap* map, int r, const float (&x)[W], int cx,
                                             int cy, bool live) {
    const uint32_t b = s.base + (uint32_t)(s.buf * STG_BYTES);
    if (s.issuer) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");  // this buffer's last store has read it
    named_sync(s.bar_id);
    if (KIND == OUT_R32) {
        const uint32_t row = b + (uint32_t)r * 64u;
#pragma unroll
        for (int k = 0; k < 4; k++)
            st_shared_v4(row + ((uint32_t)(k ^ ((r >> 1) & 3)) << 4), __float_as_uint(x[4 * k]),
                         __float_as_uint(x[4 * k + 1]), __float_as_uint(x[4 * k + 2]), __float_as_uint(x[4 * k + 3]));
    } else if (KIND == OUT_R16) {
        const uint32_t row = b + (uint32_t)r * 32u;
#pragma unroll
        for (int k = 0; k < 2; k++)
            st_shared_v4(row + ((uint32_t)(k ^ ((r >> 2) & 1)) << 4), pack_bf16(x[8 * k], x[8 * k + 1]),
                         pack_bf16(x[8 * k + 2], x[8 * k + 3]), pack_bf16(x[8 * k + 4], x[8 * k + 5]),
                         pack_bf16(x[8 * k + 6], x[8 * k + 7]));
    } else if (KIND == OUT_T32) {
#pragma unroll
        for (int j = 0; j < W; j++)
            asm volatile("st.shared.b32 [%0], %1;" ::"r"(b + (uint32_t)(j * 512 + r * 4)), "r"(__float_as_uint(x[j]))
                         : "memory");
    } else {
#pragma unroll
        for (int j = 0; j < W; j++) {
            const __nv_bfloat16 h = __float2bfloat16_rn(x[j]);
            asm volatile("st.shared.b16 [%0], %1;" ::"r"(b + (uint32_t)(j * 256 + r * 2)),
                         "h"(*reinterpret_cast<const unsigned short*>(&h))
                         : "memory");
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    named_sync(s.bar_id);
    if (s.issuer && live) {
        asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                         reinterpret_cast<uint64_t>(map)),
                     "r"(b), "r"(cx), "r"(cy)
                     : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
    s.buf ^= 1;
}

// Epilogue of one W-column chunk: rows m0 + r, columns n .. n+W-1, x = accumulator.
__device__ __forceinline__ void epilogue_chunk(const GemmArgs& g, const StoreMaps& sm, const Flags& f, Stager& st,
                                               int m0, int r, int n, float (&x)[W], bool live) {
    const int m = m0 + r;
    const bool row_ok = live && m < g.M;
    const bool full = n + W <= g.N;
    if (g.bias) {
#pragma unroll
        for (int j = 0; j < W; j++)
            if (n + j < g.N) x[j] += __ldg(g.bias + n + j);
    }
    if (g.epi == EPI_GELU) {
        if (g.pre) {
            if (f.tma_pre) {
                staged_store<OUT_R32>(st, &sm.pre, r, x, n, m0, live);
            } else if (row_ok) {
                float* p = g.pre + (int64_t)m * g.ldpre + n;
                if (full && f.vec_pre) {
#pragma unroll
                    for (int j = 0; j < W; j += 4)
                        *reinterpret_cast<float4*>(p + j) = make_float4(x[j], x[j + 1], x[j + 2], x[j + 3]);
                } else {
#pragma unroll
                    for (int j = 0; j < W; j++)
                        if (n + j < g.N) p[j] = x[j];
                }
            }
        }
#pragma unroll
        for (int j = 0; j < W; j++) x[j] = gelu_exact(x[j]);
    } else if (g.epi == EPI_GELU_GRAD) {
        if (row_ok) {
            const float* p = g.pre + (int64_t)m * g.ldpre + n;
            if (full && f.vec_pre) {
#pragma unroll
                for (int j = 0; j < W; j += 4) {
                    const float4 v = __ldg(reinterpret_cast<const float4*>(p + j));
                    x[j] *= gelu_grad(v.x);
                    x[j + 1] *= gelu_grad(v.y);
                    x[j + 2] *= gelu_grad(v.z);
                    x[j + 3] *= gelu_grad(v.w);
                }
            } else {
#pragma unroll
                for (int j = 0; j < W; j++)
                    if (n + j < g.N) x[j] *= gelu_grad(__ldg(p + j));
            }
        }
    }
#pragma unroll
    for (int j = 0; j < W; j++) x[j] *= g.alpha;
    if (g.out_f32) {
        if (f.tma_f32) {
            staged_store<OUT_R32>(st, &sm.f32, r, x, n, m0, live);
        } else if (row_ok) {
            float* o = g.out_f32 + (int64_t)m * g.ldo + n;
            if (full && f.vec_f32) {
#pragma unroll
                for (int j = 0; j < W; j += 4)
                    *reinterpret_cast<float4*>(o + j) = make_float4(x[j], x[j + 1], x[j + 2], x[j + 3]);
            } else {
#pragma unroll
                for (int j = 0; j < W; j++)
                    if (n + j < g.N) o[j] = x[j];
            }
        }
    }
    if (g.out_bf16) {
        if (f.tma_bf16) {
            staged_store<OUT_R16>(st, &sm.bf16, r, x, n, m0, live);
        } else if (row_ok) {
            __nv_bfloat16* o = g.out_bf16 + (int64_t)m * g.ldo + n;
            if (full && f.vec_bf16) {
#pragma unroll
                for (int j = 0; j < W; j += 8) {
                    uint4 v;
                    v.x = pack_bf16(x[j], x[j + 1]);
                    v.y = pack_bf16(x[j + 2], x[j + 3]);
                    v.z = pack_bf16(x[j + 4], x[j + 5]);
                    v.w = pack_bf16(x[j + 6], x[j + 7]);
                    *reinterpret_cast<uint4*>(o + j) = v;
                }
            } else {
#pragma unroll
                for (int j = 0; j < W; j++)
                    if (n + j < g.N) o[j] = __float2bfloat16_rn(x[j]);
            }
        }
    }
    // direct transposed stores: lanes hold consecutive m, so each column is one coalesced warp store
    if (g.out_t_bf16) {
        if (f.tma_tbf16) {
            staged_store<OUT_T16>(st, &sm.tbf16, r, x, m0, n, live);
        } else if (row_ok) {
#pragma unroll
            for (int j = 0; j < W; j++)
                if (n + j < g.N) g.out_t_bf16[(int64_t)(n + j) * g.ldt + m] = __float2bfloat16_rn(x[j]);
        }
    }
    if (g.out_t_f32) {
        if (f.tma_tf32) {
            staged_store<OUT_T32>(st, &sm.tf32, r, x, m0, n, live);
        } else if (row_ok) {
#pragma unroll
            for (int j = 0; j < W; j++)
                if (n + j < g.N) g.out_t_f32[(int64_t)(n + j) * g.ldt + m] = x[j];
        }
    }
}

template <int BN>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    gemm_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                const __grid_constant__ GemmArgs g, const __grid_constant__ StoreMaps sm, const Flags f) {
    using C = Cfg<BN>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t pad = ((su32(smem_raw) + 1023u) & ~1023u) - su32(smem_raw);
    unsigned char* smem = smem_raw + pad;
    const uint32_t ring = su32(smem);
    const uint32_t staging = ring + C::RING;
    const uint32_t bars = staging + C::STAGING;
    auto full_bar = [&](int s) { return bars + 8u * (uint32_t)s; };
    auto empty_bar = [&](int s) { return bars + 8u * (uint32_t)(C::STAGES + s); };
    auto tfull_bar = [&](int a) { return bars + 8u * (uint32_t)(2 * C::STAGES + a); };
    auto tempty_bar = [&](int a) { return bars + 8u * (uint32_t)(2 * C::STAGES + 2 + a); };
    const uint32_t done_bar = bars + 8u * (uint32_t)(2 * C::STAGES + 4);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::RING + C::STAGING + 8 * C::N_BAR);
    volatile uint32_t* abort = tmem_slot + 1;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles_n = (g.N + BN - 1) / BN;
    const int tiles = ((g.M + BM - 1) / BM) * n_tiles_n;
    const int nk = (g.K + BK - 1) / BK;

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "n"(C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; s++) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int a = 0; a < 2; a++) {
            mbar_init(tfull_bar(a), 1);
            mbar_init(tempty_bar(a), N_EPI_WARPS);
        }
        mbar_init(done_bar, 1);
        *abort = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_a)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_b)) : "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------------------- TMA producer
        int stage = 0;
        uint32_t phase = 0;
        uint32_t used = 0, last_par = 0;  // per stage: ever loaded / parity of its last load
        for (int t = blockIdx.x; t < tiles && !*abort; t += gridDim.x) {
            const int m0 = (t / n_tiles_n) * BM, n0 = (t % n_tiles_n) * BN;
            for (int kc = 0; kc < nk; kc++) {
                if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort, g.status)) break;
                const uint32_t a_dst = ring + (uint32_t)(stage * C::STAGE), b_dst = a_dst + C::A_BYTES;
                mbar_expect_tx(full_bar(stage), (uint32_t)C::STAGE);
                tma_load_2d(a_dst, &map_a, kc * BK, m0, full_bar(stage));
                tma_load_2d(b_dst, &map_b, kc * BK, n0, full_bar(stage));
                used |= 1u << stage;
                last_par = (last_par & ~(1u << stage)) | (phase << stage);
                if (++stage == C::STAGES) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
        }
        // let every issued copy land before the CTA may exit
        for (int s = 0; s < C::STAGES; s++)
            if (used >> s & 1u) mbar_wait(full_bar(s), last_par >> s & 1u, abort, g.status, false);
    } else if (warp == 1 && lane == 0) {
        // ---------------------------------------------------------------- MMA issuer
        constexpr uint32_t idesc = instr_desc(BN);
        int stage = 0;
        uint32_t phase = 0;
        int i = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, i++) {
            const int acc = i & 1;
            const uint32_t use = (uint32_t)(i >> 1);
            if (!mbar_wait(tempty_bar(acc), (use & 1u) ^ 1u, abort, g.status)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t d_tmem = tmem + (uint32_t)(acc * BN);
            bool ok = true;
            for (int kc = 0; kc < nk; kc++) {
                if (!mbar_wait(full_bar(stage), phase, abort, g.status)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a0 = ring + (uint32_t)(stage * C::STAGE), b0 = a0 + C::A_BYTES;
#pragma unroll
                for (int s = 0; s < BK / 16; s++) {
                    const uint64_t ad = smem_desc_sw128(a0 + (uint32_t)(s * 32));
                    const uint64_t bd = smem_desc_sw128(b0 + (uint32_t)(s * 32));
                    const uint32_t accumulate = (kc > 0 || s > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
                        : "memory");
                }
                mma_commit(empty_bar(stage));  // the stage is free once these MMAs have read it
                if (++stage == C::STAGES) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
            if (!ok) break;
            mma_commit(tfull_bar(acc));
        }
        // every MMA issued has completed before TMEM is released
        mma_commit(done_bar);
        mbar_wait(done_bar, 0u, abort, g.status, false);
    } else if (warp >= 2) {
        // ---------------------------------------------------------------- epilogue
        // Every thread of a column group runs the same sequence of chunks and
        // staged stores (their named barriers must match), also after an abort,
        // when it skips the TMEM reads and the stores themselves.
        const int q = warp & 3;              // TMEM lane quarter this warp may access
        const int grp = (warp - 2) >> 2;     // column group: columns [grp, grp + 1) * BN / EPI_GROUPS
        const int r = 32 * q + lane;         // row within the tile
        Stager st;
        st.base = staging + (uint32_t)(grp * 2 * STG_BYTES);
        st.buf = 0;
        st.bar_id = 1 + grp;
        st.issuer = ((warp - 2) & 3) == 0 && lane == 0;
        constexpr int COLS = BN / EPI_GROUPS;
        int i = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, i++) {
            const int acc = i & 1;
            const uint32_t use = (uint32_t)(i >> 1);
            int ok = 1;
            if (lane == 0) ok = mbar_wait(tfull_bar(acc), use & 1u, abort, g.status) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int m0 = (t / n_tiles_n) * BM, n0 = (t % n_tiles_n) * BN;
            for (int c = grp * COLS; c < (grp + 1) * COLS; c += W) {
                if (n0 + c >= g.N) break;
                float x[W];
                if (ok) {
                    uint32_t v[W];
                    const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * BN + c);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                        "%12, %13, %14, %15}, [%16];"
                        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                          "=r"(v[14]), "=r"(v[15])
                        : "r"(taddr));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int j = 0; j < W; j++) x[j] = __uint_as_float(v[j]);
                } else {
#pragma unroll
                    for (int j = 0; j < W; j++) x[j] = 0.0f;
                }
                epilogue_chunk(g, sm, f, st, m0, r, n0 + c, x, ok != 0 && !*abort);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty_bar(acc));
        }
        if (st.issuer) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(C::TMEM_COLS)
                     : "memory");
}

bool encode(CUtensorMap* map, const void* base, CUtensorMapDataType dt, int esize, int64_t rows, int64_t cols,
            int64_t ld, int box_cols, int box_rows, CUtensorMapSwizzle sw) {
    return encode_2d(map, base, dt, esize, rows, cols, ld, box_cols, box_rows, sw);
}

// Operand map: K-major bf16 [rows][ld]; box = 64 K-elements (128 B) x box_rows, written to shared
// memory with the 128-byte swizzle.
bool make_map(CUtensorMap* map, const __nv_bfloat16* base, int rows, int K, int64_t ld, int box_rows) {
    return encode(map, base, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, rows, K, ld, BK, box_rows,
                  CU_TENSOR_MAP_SWIZZLE_128B);
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

template <int BN>
cudaError_t gemm_launch(const GemmArgs& g, int sms, cudaStream_t s) {
    using C = Cfg<BN>;
    static PerDeviceOnce once;  // the shared-memory opt-in holds per device
    const cudaError_t attr = once.run(
        [] { return cudaFuncSetAttribute(gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM); });
    if (attr != cudaSuccess) return attr;
    CUtensorMap ma, mb;
    if (!make_map(&ma, g.A, g.M, g.K, g.lda, BM) || !make_map(&mb, g.B, g.N, g.K, g.ldb, BN))
        return cudaErrorInvalidValue;
    Flags f;
    f.vec_f32 = aligned16(g.out_f32) && g.ldo % 4 == 0;
    f.vec_bf16 = aligned16(g.out_bf16) && g.ldo % 8 == 0;
    f.vec_pre = aligned16(g.pre) && g.ldpre % 4 == 0;
    // Staged TMA stores wherever the output's base and row stride are 16-byte aligned.
    StoreMaps sm;
    memset(&sm, 0, sizeof(sm));
    const auto F32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const auto B16 = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    f.tma_pre = g.epi == EPI_GELU && f.vec_pre &&
                encode(&sm.pre, g.pre, F32, 4, g.M, g.N, g.ldpre, W, BM, CU_TENSOR_MAP_SWIZZLE_64B);
    f.tma_f32 = f.vec_f32 && encode(&sm.f32, g.out_f32, F32, 4, g.M, g.N, g.ldo, W, BM, CU_TENSOR_MAP_SWIZZLE_64B);
    f.tma_bf16 = f.vec_bf16 && encode(&sm.bf16, g.out_bf16, B16, 2, g.M, g.N, g.ldo, W, BM, CU_TENSOR_MAP_SWIZZLE_32B);
    f.tma_tbf16 = aligned16(g.out_t_bf16) && g.ldt % 8 == 0 &&
                  encode(&sm.tbf16, g.out_t_bf16, B16, 2, g.N, g.M, g.ldt, BM, W, CU_TENSOR_MAP_SWIZZLE_NONE);
    f.tma_tf32 = aligned16(g.out_t_f32) && g.ldt % 4 == 0 &&
                 encode(&sm.tf32, g.out_t_f32, F32, 4, g.N, g.M, g.ldt, BM, W, CU_TENSOR_MAP_SWIZZLE_NONE);
    const int tiles = ((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN);
    const int grid = tiles < sms ? tiles : sms;
    gemm_kernel<BN><<<grid, GEMM_THREADS, C::SMEM, s>>>(ma, mb, g, sm, f);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gemm_bf16(const GemmArgs& g, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0 || g.K <= 0) return cudaSuccess;
    if ((g.lda % 8) || (g.ldb % 8) || ((uintptr_t)g.A & 15) || ((uintptr_t)g.B & 15) || g.lda < g.K ||
        g.ldb < g.K)
        return cudaErrorInvalidValue;
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
        return cudaErrorInvalidDevice;
    // Widest tile that still gives every SM a tile; narrower tiles for short, long-K products.
    const int mt = (g.M + BM - 1) / BM;
    auto tiles = [&](int bn) { return mt * ((g.N + bn - 1) / bn); };
    if (g.N > 128 && tiles(256) >= sms) return gemm_launch<256>(g, sms, s);
    if (g.N > 64 && tiles(128) >= sms) return gemm_launch<128>(g, sms, s);
    return gemm_launch<64>(g, sms, s);
}

}  // namespace sat

// ------------------------------------------------------------------ C ABI --
#include "../../include/satsampler.h"
#include "host.hpp"

extern "C" sat_status sat_gemm_bf16(int32_t M, int32_t N, int32_t K, const void* A, int64_t lda, const void* B,
                                    int64_t ldb, const float* bias, int32_t epilogue, float* pre, int64_t ldpre,
                                    float alpha, float* out_f32, void* out_bf16, int64_t ldo, void* out_t_bf16,
                                    float* out_t_f32, int64_t ldt, uint32_t* status, void* stream) {
    if (M < 0 || N < 0 || K < 0 || epilogue < 0 || epilogue > 2) return sat::report_error(SAT_ERR_ARG, "bad GEMM shape");
    if (M == 0 || N == 0 || K == 0) return SAT_OK;
    if (!A || !B || lda < K || ldb < K || (lda % 8) || (ldb % 8) || ((uintptr_t)A & 15) || ((uintptr_t)B & 15))
        return sat::report_error(SAT_ERR_ARG, "A/B must be 16-byte aligned with leading dimensions >= K, multiples of 8");
    if (epilogue == sat::EPI_GELU_GRAD && !pre) return sat::report_error(SAT_ERR_ARG, "GELU-gradient epilogue needs pre");
    if (((out_f32 || out_bf16) && ldo < N) || ((out_t_bf16 || out_t_f32) && ldt < M) || (pre && ldpre < N))
        return sat::report_error(SAT_ERR_ARG, "output leading dimension too small");
    if (!status) return sat::report_error(SAT_ERR_ARG, "status word is NULL");
    sat::GemmArgs g;
    g.M = M; g.N = N; g.K = K;
    g.A = (const __nv_bfloat16*)A; g.lda = lda;
    g.B = (const __nv_bfloat16*)B; g.ldb = ldb;
    g.bias = bias; g.epi = epilogue; g.pre = pre; g.ldpre = ldpre; g.alpha = alpha;
    g.out_f32 = out_f32; g.out_bf16 = (__nv_bfloat16*)out_bf16; g.ldo = ldo;
    g.out_t_bf16 = (__nv_bfloat16*)out_t_bf16; g.out_t_f32 = out_t_f32; g.ldt = ldt;
    g.status = (unsigned int*)status;
    cudaError_t e = sat::launch_gemm_bf16(g, (cudaStream_t)stream);
    if (e != cudaSuccess) return sat::report_error(SAT_ERR_CUDA, std::string("gemm: ") + cudaGetErrorString(e));
    return SAT_OK;
}
