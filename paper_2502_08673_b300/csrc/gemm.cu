// Dense BF16 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a) with a
// fused epilogue, for the proposal network's layers.
//
//   D[m][n] = sum_k A[m][k] * B[n][k]      (A: [M][lda], B: [N][ldb], both K-major bf16)
//   out = epi(D + bias[n])                 (epi: identity / GELU / times GELU'(Z[m][n]))
//
// One CTA computes a 128 x BN tile (BN = 64, 128 or 256) with one tcgen05.mma
// per 16-deep K slice, issued by a single thread; operands are staged by
// cp.async in the canonical no-swizzle K-major layout (8-row x 16-byte core
// matrices; core matrices adjacent in K are 128 B apart, 8-row groups 1 KB
// apart), double-buffered over 64-deep K chunks; the FP32 accumulator lives in
// tensor memory and is read back with tcgen05.ld for the epilogue.  Every
// mbarrier wait is bounded and records a status bit instead of hanging.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "gemm.hpp"

namespace sat {
namespace {

constexpr int BM = 128;
constexpr int BK = 64;                  // K chunk per stage (bf16: 128 B per row)
constexpr int GEMM_THREADS = 128;       // 4 warps: warp w owns TMEM lanes 32w .. 32w+31
constexpr uint32_t GEMM_WAIT_LIMIT = 1u << 26;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp16_zfill(void* smem, const void* gmem, bool valid) {
    const uint32_t n = valid ? 16u : 0u;  // 0 source bytes: the 16 destination bytes are zero-filled
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(su32(smem)), "l"(gmem), "r"(n) : "memory");
}

// Canonical no-swizzle K-major matrix descriptor: start, LBO (K step between
// core matrices) = 128 B, SBO (8-row step) = 1024 B, version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(128u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
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

// Smem offset of the 16-byte piece c (0..7) of row r of a K-major chunk.
__device__ __forceinline__ uint32_t piece_off(int r, int c) { return (uint32_t)((r >> 3) * 1024 + c * 128 + (r & 7) * 16); }

template <int BN>
__global__ void __launch_bounds__(GEMM_THREADS) gemm_kernel(GemmArgs g) {
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2, STAGE = A_BYTES + B_BYTES;
    unsigned char* stage_buf[2] = {smem, smem + STAGE};
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * STAGE);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 2 * STAGE + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "n"(BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const int nk = (g.K + BK - 1) / BK;
    auto load_chunk = [&](int kc, unsigned char* buf) {
        const int k0 = kc * BK;
        for (int i = tid; i < BM * 8; i += GEMM_THREADS) {
            const int r = i >> 3, c = i & 7, m = m0 + r, k = k0 + c * 8;
            const bool ok = m < g.M && k < g.K;
            cp16_zfill(buf + piece_off(r, c), ok ? (const void*)(g.A + (int64_t)m * g.lda + k) : (const void*)g.A, ok);
        }
        for (int i = tid; i < BN * 8; i += GEMM_THREADS) {
            const int r = i >> 3, c = i & 7, n = n0 + r, k = k0 + c * 8;
            const bool ok = n < g.N && k < g.K;
            cp16_zfill(buf + A_BYTES + piece_off(r, c), ok ? (const void*)(g.B + (int64_t)n * g.ldb + k) : (const void*)g.B,
                       ok);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    uint32_t phase = 0;
    bool timeout = false;
    auto wait_mma = [&]() {
        uint32_t it = 0, ok = 0;
        while (!timeout) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 1000000;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(ok)
                : "r"(su32(bar)), "r"(phase)
                : "memory");
            if (ok) break;
            if (++it >= GEMM_WAIT_LIMIT) {
                timeout = true;
                if (tid == 0) atomicOr(g.status, 8u);
            }
        }
        phase ^= 1u;
    };
    // At most one commit is outstanding on the barrier at any time, so the
    // parity wait always targets the phase of that commit.
    load_chunk(0, stage_buf[0]);
    for (int kc = 0; kc < nk; kc++) {
        unsigned char* buf = stage_buf[kc & 1];
        if (kc >= 1) wait_mma();  // chunk kc-1's MMAs are done: its buffer is free
        if (kc + 1 < nk) {
            load_chunk(kc + 1, stage_buf[(kc + 1) & 1]);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = su32(buf), b0 = su32(buf + A_BYTES);
#pragma unroll
            for (int s = 0; s < BK / 16; s++) {
                const uint64_t ad = smem_desc(a0 + s * 256), bd = smem_desc(b0 + s * 256);
                const uint32_t acc = (kc > 0 || s > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(instr_desc(BN)), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                         : "memory");
        }
        __syncthreads();
    }
    wait_mma();  // the last chunk's commit
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue: thread owns row m = m0 + 32 warp + lane (TMEM lane), 16 columns per load
    const int m = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t r[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (m >= g.M || timeout) continue;
#pragma unroll
        for (int j = 0; j < 16; j++) {
            const int n = n0 + c0 + j;
            if (n >= g.N) break;
            float x = __uint_as_float(r[j]);
            if (g.bias) x += g.bias[n];
            if (g.epi == EPI_GELU) {
                if (g.pre) g.pre[(int64_t)m * g.ldpre + n] = x;
                x = gelu_exact(x);
            } else if (g.epi == EPI_GELU_GRAD) {
                x *= gelu_grad(g.pre[(int64_t)m * g.ldpre + n]);
            }
            x *= g.alpha;
            if (g.out_f32) g.out_f32[(int64_t)m * g.ldo + n] = x;
            if (g.out_bf16) g.out_bf16[(int64_t)m * g.ldo + n] = __float2bfloat16_rn(x);
            if (g.out_t_bf16) g.out_t_bf16[(int64_t)n * g.ldt + m] = __float2bfloat16_rn(x);
            if (g.out_t_f32) g.out_t_f32[(int64_t)n * g.ldt + m] = x;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(BN) : "memory");
}

template <int BN>
cudaError_t gemm_launch(const GemmArgs& g, cudaStream_t s) {
    constexpr int smem = 2 * (BM * BK * 2 + BN * BK * 2) + 64;
    static cudaError_t attr = cudaFuncSetAttribute(gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (attr != cudaSuccess) return attr;
    dim3 grid((unsigned)((g.N + BN - 1) / BN), (unsigned)((g.M + BM - 1) / BM));
    gemm_kernel<BN><<<grid, GEMM_THREADS, smem, s>>>(g);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gemm_bf16(const GemmArgs& g, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0 || g.K <= 0) return cudaSuccess;
    if ((g.lda % 8) || (g.ldb % 8) || ((uintptr_t)g.A & 15) || ((uintptr_t)g.B & 15)) return cudaErrorInvalidValue;
    if (g.N <= 64) return gemm_launch<64>(g, s);
    if (g.N <= 128) return gemm_launch<128>(g, s);
    return gemm_launch<256>(g, s);
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
