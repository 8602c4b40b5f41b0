// Internal BF16 tensor-core GEMM with fused epilogue (see gemm.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace sat {

enum GemmEpi { EPI_NONE = 0, EPI_GELU = 1, EPI_GELU_GRAD = 2 };

struct GemmArgs {
    int M = 0, N = 0, K = 0;
    const __nv_bfloat16* A = nullptr;   // [M][lda], K-major
    int64_t lda = 0;
    const __nv_bfloat16* B = nullptr;   // [N][ldb], K-major
    int64_t ldb = 0;
    const float* bias = nullptr;        // [N] or null
    int epi = EPI_NONE;
    float* pre = nullptr;               // EPI_GELU: stores D + bias (may be null); EPI_GELU_GRAD: reads it
    int64_t ldpre = 0;
    float alpha = 1.0f;                 // final scale
    float* out_f32 = nullptr;           // [M][ldo]
    __nv_bfloat16* out_bf16 = nullptr;  // [M][ldo]
    int64_t ldo = 0;
    __nv_bfloat16* out_t_bf16 = nullptr;  // [N][ldt] (transposed store)
    float* out_t_f32 = nullptr;           // [N][ldt]
    int64_t ldt = 0;
    unsigned int* status = nullptr;     // bit 3: a bounded wait expired
};

cudaError_t launch_gemm_bf16(const GemmArgs& g, cudaStream_t s);

}  // namespace sat
