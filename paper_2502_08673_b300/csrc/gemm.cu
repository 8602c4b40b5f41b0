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
//   warps 2..9  epilogue: tcgen05.ld of the finished accumulator, bias /
//               activation / scale, 16-byte stores.
// Two TMEM accumulators alternate between tiles, so the epilogue of tile i
// runs while the MMAs of tile i+1 execute.  Operands sit in shared memory in
// the canonical no-swizzle K-major layout, written directly by TMA: one box of
// 8 K-elements (16 bytes) x rows per 8-column group, so a core matrix (8 rows x
// 16 B) is contiguous, 8-row groups are 128 B apart and adjacent K groups are
// rows x 16 B apart.  Out-of-range rows and K columns are zero-filled by TMA.
// Every mbarrier wait is bounded in time; an expired wait sets bit 3 of the
// status word and every role of the CTA stops, after letting its own copies
// and MMAs in flight finish.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "gemm.hpp"

namespace sat {
namespace {

constexpr int BM = 128;
constexpr int BK = 64;                               // K elements per stage: 8 groups of 16 bytes
constexpr int N_EPI_WARPS = 8;                       // two per TMEM lane quarter, one per half of the columns
constexpr int GEMM_THREADS = 64 + 32 * N_EPI_WARPS;  // + producer warp + MMA warp
constexpr uint64_t WAIT_NS = 2000000000ull;          // bound of one mbarrier wait (2 s)

template <int BN>
struct Cfg {
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;  // a multiple of 1024
    static constexpr int STAGES = BN == 256 ? 4 : (BN == 128 ? 6 : 8);
    static constexpr int RING = STAGES * STAGE;
    // barriers: full[STAGES], empty[STAGES], tmem_full[2], tmem_empty[2], done
    static constexpr int N_BAR = 2 * STAGES + 5;
    static constexpr int SMEM = 1024 + RING + 8 * N_BAR + 16;  // + slack to align the ring to 1 KB
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

// No-swizzle K-major shared-memory matrix descriptor: start address, LBO = step
// between core matrices adjacent in K, SBO = step between 8-row groups,
// descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;
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
    bool vec_f32, vec_bf16, vec_pre;  // row-major outputs / pre allow 16-byte accesses
};

// Epilogue of one 32-column chunk of row m (columns n .. n+31), x = accumulator.
__device__ __forceinline__ void epilogue_chunk(const GemmArgs& g, Flags f, int m, int n, float (&x)[32]) {
    const bool row_ok = m < g.M;
    const bool full = n + 32 <= g.N;
    if (g.bias) {
#pragma unroll
        for (int j = 0; j < 32; j++)
            if (n + j < g.N) x[j] += __ldg(g.bias + n + j);
    }
    if (g.epi == EPI_GELU) {
        if (g.pre && row_ok) {
            float* p = g.pre + (int64_t)m * g.ldpre + n;
            if (full && f.vec_pre) {
#pragma unroll
                for (int j = 0; j < 32; j += 4)
                    *reinterpret_cast<float4*>(p + j) = make_float4(x[j], x[j + 1], x[j + 2], x[j + 3]);
            } else {
#pragma unroll
                for (int j = 0; j < 32; j++)
                    if (n + j < g.N) p[j] = x[j];
            }
        }
#pragma unroll
        for (int j = 0; j < 32; j++) x[j] = gelu_exact(x[j]);
    } else if (g.epi == EPI_GELU_GRAD) {
        if (row_ok) {
            const float* p = g.pre + (int64_t)m * g.ldpre + n;
            if (full && f.vec_pre) {
#pragma unroll
                for (int j = 0; j < 32; j += 4) {
                    const float4 v = __ldg(reinterpret_cast<const float4*>(p + j));
                    x[j] *= gelu_grad(v.x);
                    x[j + 1] *= gelu_grad(v.y);
                    x[j + 2] *= gelu_grad(v.z);
                    x[j + 3] *= gelu_grad(v.w);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 32; j++)
                    if (n + j < g.N) x[j] *= gelu_grad(__ldg(p + j));
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 32; j++) x[j] *= g.alpha;
    if (row_ok && g.out_f32) {
        float* o = g.out_f32 + (int64_t)m * g.ldo + n;
        if (full && f.vec_f32) {
#pragma unroll
            for (int j = 0; j < 32; j += 4)
                *reinterpret_cast<float4*>(o + j) = make_float4(x[j], x[j + 1], x[j + 2], x[j + 3]);
        } else {
#pragma unroll
            for (int j = 0; j < 32; j++)
                if (n + j < g.N) o[j] = x[j];
        }
    }
    if (row_ok && g.out_bf16) {
        __nv_bfloat16* o = g.out_bf16 + (int64_t)m * g.ldo + n;
        if (full && f.vec_bf16) {
#pragma unroll
            for (int j = 0; j < 32; j += 8) {
                uint4 v;
                __nv_bfloat162 h0 = __floats2bfloat162_rn(x[j], x[j + 1]), h1 = __floats2bfloat162_rn(x[j + 2], x[j + 3]);
                __nv_bfloat162 h2 = __floats2bfloat162_rn(x[j + 4], x[j + 5]), h3 = __floats2bfloat162_rn(x[j + 6], x[j + 7]);
                v.x = *reinterpret_cast<uint32_t*>(&h0);
                v.y = *reinterpret_cast<uint32_t*>(&h1);
                v.z = *reinterpret_cast<uint32_t*>(&h2);
                v.w = *reinterpret_cast<uint32_t*>(&h3);
                *reinterpret_cast<uint4*>(o + j) = v;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 32; j++)
                if (n + j < g.N) o[j] = __float2bfloat16_rn(x[j]);
        }
    }
    // transposed stores: lanes hold consecutive m, so each column is one coalesced warp store
    if (row_ok && g.out_t_bf16) {
#pragma unroll
        for (int j = 0; j < 32; j++)
            if (n + j < g.N) g.out_t_bf16[(int64_t)(n + j) * g.ldt + m] = __float2bfloat16_rn(x[j]);
    }
    if (row_ok && g.out_t_f32) {
#pragma unroll
        for (int j = 0; j < 32; j++)
            if (n + j < g.N) g.out_t_f32[(int64_t)(n + j) * g.ldt + m] = x[j];
    }
}

template <int BN>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    gemm_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                const __grid_constant__ GemmArgs g, const Flags f) {
    using C = Cfg<BN>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t pad = ((su32(smem_raw) + 1023u) & ~1023u) - su32(smem_raw);
    unsigned char* smem = smem_raw + pad;
    const uint32_t ring = su32(smem);
    const uint32_t bars = ring + C::RING;
    auto full_bar = [&](int s) { return bars + 8u * (uint32_t)s; };
    auto empty_bar = [&](int s) { return bars + 8u * (uint32_t)(C::STAGES + s); };
    auto tfull_bar = [&](int a) { return bars + 8u * (uint32_t)(2 * C::STAGES + a); };
    auto tempty_bar = [&](int a) { return bars + 8u * (uint32_t)(2 * C::STAGES + 2 + a); };
    const uint32_t done_bar = bars + 8u * (uint32_t)(2 * C::STAGES + 4);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::RING + 8 * C::N_BAR);
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
#pragma unroll
                for (int c = 0; c < BK / 8; c++) {
                    tma_load_2d(a_dst + (uint32_t)(c * BM * 16), &map_a, kc * BK + 8 * c, m0, full_bar(stage));
                    tma_load_2d(b_dst + (uint32_t)(c * BN * 16), &map_b, kc * BK + 8 * c, n0, full_bar(stage));
                }
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
                    const uint64_t ad = smem_desc(a0 + (uint32_t)(s * 2 * BM * 16), BM * 16, 128);
                    const uint64_t bd = smem_desc(b0 + (uint32_t)(s * 2 * BN * 16), BN * 16, 128);
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
        const int q = warp & 3;              // TMEM lane quarter this warp may access
        const int half = (warp - 2) >> 2;    // which half of the tile's columns
        int i = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, i++) {
            const int acc = i & 1;
            const uint32_t use = (uint32_t)(i >> 1);
            int ok = 1;
            if (lane == 0) ok = mbar_wait(tfull_bar(acc), use & 1u, abort, g.status) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int m = (t / n_tiles_n) * BM + 32 * q + lane, n0 = (t % n_tiles_n) * BN;
            for (int c = half * (BN / 2); c < (half + 1) * (BN / 2); c += 32) {
                if (n0 + c >= g.N) break;
                uint32_t r[32];
                const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * BN + c);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                    "[%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                      "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                      "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                float x[32];
#pragma unroll
                for (int j = 0; j < 32; j++) x[j] = __uint_as_float(r[j]);
                epilogue_chunk(g, f, m, n0 + c, x);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty_bar(acc));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(C::TMEM_COLS)
                     : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// 2-D map over a K-major bf16 matrix [rows][ld] (K contiguous); box = 8 K-elements x box_rows.
bool make_map(CUtensorMap* map, const __nv_bfloat16* base, int rows, int K, int64_t ld, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {8u, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1u, 1u};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

template <int BN>
cudaError_t gemm_launch(const GemmArgs& g, int sms, cudaStream_t s) {
    using C = Cfg<BN>;
    static cudaError_t attr =
        cudaFuncSetAttribute(gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (attr != cudaSuccess) return attr;
    CUtensorMap ma, mb;
    if (!make_map(&ma, g.A, g.M, g.K, g.lda, BM) || !make_map(&mb, g.B, g.N, g.K, g.ldb, BN))
        return cudaErrorInvalidValue;
    Flags f;
    f.vec_f32 = aligned16(g.out_f32) && g.ldo % 4 == 0;
    f.vec_bf16 = aligned16(g.out_bf16) && g.ldo % 8 == 0;
    f.vec_pre = aligned16(g.pre) && g.ldpre % 4 == 0;
    const int tiles = ((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN);
    const int grid = tiles < sms ? tiles : sms;
    gemm_kernel<BN><<<grid, GEMM_THREADS, C::SMEM, s>>>(ma, mb, g, f);
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
