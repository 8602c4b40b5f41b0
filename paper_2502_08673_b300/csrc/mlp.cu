// Learned proposal network: an MLP from Gaussian noise z (n_in) to initial
// logits of the primary inputs (n_out), z -> GELU(W1 z + b1) -> GELU(W2 . + b2)
// -> W3 . + b3, trained with implicit maximum likelihood (IMLE: for every
// training solution, the nearest of K noise candidates under the summed BCE is
// pulled towards it).  Weights: FP32 masters, BF16 copies (and transposed
// copies for the input-gradient GEMMs); activations BF16; every layer is a
// tcgen05 GEMM (gemm.cu) with FP32 accumulation.  The paper has no learned
// component: this is the library's proposal option.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/satsampler.h"
#include "gemm.hpp"
#include "host.hpp"

struct sat_mlp {
    int device = 0;
    int n_in = 0, h = 0, n_out = 0, n_out_p = 0;
    int64_t cap = 0;
    uint64_t np = 0;
    uint64_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
    float *P = nullptr, *G = nullptr, *M1 = nullptr, *M2 = nullptr;
    __nv_bfloat16 *W1b = nullptr, *W2b = nullptr, *W3b = nullptr, *W2Tb = nullptr, *W3Tb = nullptr;
    __nv_bfloat16 *Z = nullptr, *ZT = nullptr, *Zc = nullptr;
    float *pre1 = nullptr, *pre2 = nullptr, *Y = nullptr;
    __nv_bfloat16 *H1 = nullptr, *H1T = nullptr, *H2 = nullptr, *H2T = nullptr;
    __nv_bfloat16 *dY = nullptr, *dYT = nullptr, *dA2 = nullptr, *dA2T = nullptr, *dA1 = nullptr, *dA1T = nullptr;
    float *dist = nullptr, *loss_part = nullptr;
    int32_t* choice = nullptr;
    unsigned int* status = nullptr;
    int32_t t = 0;  // Adam step count
    std::vector<void*> allocs;
};

namespace {

using bf16 = __nv_bfloat16;

// Plain view of the parameters that the weight-refresh kernel needs.
struct MlpView {
    int n_in, h, n_out, n_out_p;
    uint64_t oW1, oW2, oW3;
    const float* P;
    bf16 *W1b, *W2b, *W3b, *W2Tb, *W3Tb;
};

MlpView view_of(const sat_mlp* m) {
    MlpView v;
    v.n_in = m->n_in; v.h = m->h; v.n_out = m->n_out; v.n_out_p = m->n_out_p;
    v.oW1 = m->oW1; v.oW2 = m->oW2; v.oW3 = m->oW3; v.P = m->P;
    v.W1b = m->W1b; v.W2b = m->W2b; v.W3b = m->W3b; v.W2Tb = m->W2Tb; v.W3Tb = m->W3Tb;
    return v;
}

__device__ __forceinline__ uint4 philox(uint4 ctr, uint2 key) {
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

// z[r][4c + i] ~ N(0, 1), i = 0..3: one Philox4x32-10 block at counter (r, c, round, 1)
// gives two Box-Muller pairs, (x, y) -> i = 0, 1 (cos, sin) and (z, w) -> i = 2, 3;
// rounded to bf16.
__global__ void noise_kernel(uint64_t seed, uint32_t round, int64_t rows, int n_in, bf16* z) {
    const uint32_t groups = (uint32_t)(n_in + 3) / 4u;
    const int64_t n = rows * groups;
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        uint32_t r, c;
        if (n <= 0x7fffffff) {  // 32-bit index arithmetic whenever it suffices
            r = (uint32_t)k / groups;
            c = (uint32_t)k - r * groups;
        } else {
            r = (uint32_t)(k / groups);
            c = (uint32_t)(k % groups);
        }
        const uint4 o = philox(make_uint4(r, c, round, 1u), key);
        float g[4];
        {
            const float u1 = (float)((o.x >> 8) + 1u) * (1.0f / 16777216.0f);
            const float u2 = (float)(o.y >> 8) * (1.0f / 16777216.0f);
            const float rad = sqrtf(-2.0f * logf(u1));
            float sn, cs;
            sincospif(2.0f * u2, &sn, &cs);
            g[0] = rad * cs;
            g[1] = rad * sn;
        }
        {
            const float u1 = (float)((o.z >> 8) + 1u) * (1.0f / 16777216.0f);
            const float u2 = (float)(o.w >> 8) * (1.0f / 16777216.0f);
            const float rad = sqrtf(-2.0f * logf(u1));
            float sn, cs;
            sincospif(2.0f * u2, &sn, &cs);
            g[2] = rad * cs;
            g[3] = rad * sn;
        }
        bf16* zr = z + (int64_t)r * n_in + 4 * c;
        if (4 * (int)c + 4 <= n_in && (n_in & 3) == 0 && ((uintptr_t)z & 7) == 0) {
            __nv_bfloat162 lo = __floats2bfloat162_rn(g[0], g[1]), hi = __floats2bfloat162_rn(g[2], g[3]);
            uint2 v;
            v.x = *reinterpret_cast<uint32_t*>(&lo);
            v.y = *reinterpret_cast<uint32_t*>(&hi);
            *reinterpret_cast<uint2*>(zr) = v;
        } else {
            for (int i = 0; i < 4 && 4 * (int)c + i < n_in; i++) zr[i] = __float2bfloat16_rn(g[i]);
        }
    }
}

// bf16 weight copies: W1b, W2b, W3b row-major; W2Tb [h][h] and W3Tb [h][n_out_p] transposed (padding zero).
__global__ void refresh_kernel(MlpView m) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n1 = (int64_t)m.h * m.n_in, n2 = (int64_t)m.h * m.h, n3 = (int64_t)m.n_out * m.h;
    const int64_t n3t = (int64_t)m.h * m.n_out_p;
    if (t < n1) m.W1b[t] = __float2bfloat16_rn(m.P[m.oW1 + t]);
    if (t < n2) {
        m.W2b[t] = __float2bfloat16_rn(m.P[m.oW2 + t]);
        const int64_t n = t / m.h, k = t % m.h;  // W2[n][k] -> W2T[k][n]
        m.W2Tb[k * m.h + n] = __float2bfloat16_rn(m.P[m.oW2 + t]);
    }
    if (t < n3) m.W3b[t] = __float2bfloat16_rn(m.P[m.oW3 + t]);
    if (t < n3t) {
        const int64_t k = t / m.n_out_p, n = t % m.n_out_p;  // W3T[k][n] = W3[n][k]
        m.W3Tb[t] = n < m.n_out ? __float2bfloat16_rn(m.P[m.oW3 + n * m.h + k]) : __float2bfloat16_rn(0.0f);
    }
}

__device__ __forceinline__ float bce_term(float y, float t) {
    return fmaxf(y, 0.0f) - t * y + log1pf(expf(-fabsf(y)));
}

__device__ __forceinline__ float key_bit(const uint32_t* keys, int kw, int64_t s, int i) {
    return (float)((keys[s * kw + (i >> 5)] >> (i & 31)) & 1u);
}

// dist[c] = sum_i BCE(Y[c][i], bit i of target c / K); one warp per row, fixed lane order.
__global__ void imle_dist_kernel(const float* Y, int n_out, const uint32_t* keys, int kw, int K, int64_t rows,
                                 float* dist) {
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= rows) return;
    const int64_t s = c / K;
    float acc = 0.0f;
    for (int i = lane; i < n_out; i += 32) acc += bce_term(Y[c * n_out + i], key_bit(keys, kw, s, i));
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) dist[c] = acc;
}

// choice[s] = first argmin over its K candidates; Z[s] = Zc[s*K + choice]; ZT[j][s] = Z[s][j].
__global__ void imle_choose_kernel(const float* dist, int K, int64_t S, const bf16* Zc, int n_in, bf16* Z, bf16* ZT,
                                   int64_t ldt, int32_t* choice) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    int best = 0;
    float bd = dist[s * K];
    for (int k = 1; k < K; k++)
        if (dist[s * K + k] < bd) {
            bd = dist[s * K + k];
            best = k;
        }
    choice[s] = best;
    for (int j = 0; j < n_in; j++) {
        const bf16 v = Zc[(s * K + best) * n_in + j];
        Z[s * n_in + j] = v;
        ZT[(int64_t)j * ldt + s] = v;
    }
}

// ZT[j][s] = Z[s][j]
__global__ void transpose_z_kernel(const bf16* Z, int64_t S, int n_in, bf16* ZT, int64_t ldt) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S * n_in) return;
    const int64_t s = k / n_in, j = k % n_in;
    ZT[j * ldt + s] = Z[k];
}

// dY = (sigmoid(Y) - t) * scale as bf16, row-major [S][n_out_p] (padding 0) and
// transposed [n_out][ldt]; per-block partial sums of the BCE terms.
__global__ void bce_grad_kernel(const float* Y, int n_out, int n_out_p, const uint32_t* keys, int kw, int64_t S,
                                float scale, bf16* dY, bf16* dYT, int64_t ldt, float* loss_part) {
    __shared__ float tile[32][33];
    __shared__ float red[256];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    const int64_t s0 = (int64_t)blockIdx.y * 32;
    const int i0 = blockIdx.x * 32;
    float part = 0.0f;
    for (int r = ty; r < 32; r += 8) {
        const int64_t s = s0 + r;
        const int i = i0 + tx;
        float g = 0.0f;
        if (s < S && i < n_out) {
            const float y = Y[s * n_out + i], t = key_bit(keys, kw, s, i);
            part += bce_term(y, t);
            g = (1.0f / (1.0f + expf(-y)) - t) * scale;
        }
        if (s < S && i < n_out_p) dY[s * n_out_p + i] = __float2bfloat16_rn(g);
        tile[r][tx] = g;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int i = i0 + r;
        const int64_t s = s0 + tx;
        if (i < n_out && s < S) dYT[(int64_t)i * ldt + s] = __float2bfloat16_rn(tile[tx][r]);
    }
    red[threadIdx.x] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.0f;
        for (int k = 0; k < 256; k++) a += red[k];
        loss_part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = a;
    }
}

// out[n] = sum over rows of X[r][n] (bf16 [S][ld]), fixed row order.
__global__ void colsum_kernel(const bf16* X, int64_t S, int N, int64_t ld, float* out) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float a = 0.0f;
    for (int64_t r = 0; r < S; r++) a += __bfloat162float(X[r * ld + n]);
    out[n] = a;
}

__global__ void adam_kernel(float* P, const float* G, float* M1, float* M2, uint64_t n, float lr, float b1, float b2,
                            float eps, float step_size, float bc2s) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = G[i];
    const float m = fmaf(1.0f - b1, g - M1[i], M1[i]);
    const float v = fmaf(b2, M2[i], (1.0f - b2) * g * g);
    M1[i] = m;
    M2[i] = v;
    P[i] -= step_size * (m / (sqrtf(v) / bc2s + eps));
    (void)lr;
}

unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t gemm(int M, int N, int K, const bf16* A, int64_t lda, const bf16* B, int64_t ldb, const float* bias, int epi,
                 float* pre, int64_t ldpre, float alpha, float* of, bf16* ob, int64_t ldo, bf16* otb, float* otf,
                 int64_t ldt, unsigned* status, cudaStream_t s) {
    sat::GemmArgs g;
    g.M = M; g.N = N; g.K = K; g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.bias = bias; g.epi = epi;
    g.pre = pre; g.ldpre = ldpre; g.alpha = alpha; g.out_f32 = of; g.out_bf16 = ob; g.ldo = ldo;
    g.out_t_bf16 = otb; g.out_t_f32 = otf; g.ldt = ldt; g.status = status;
    return sat::launch_gemm_bf16(g, s);
}

// Layers 1-2 on rows Z [R][n_in]; training stores pre-activations and transposed copies.
cudaError_t hidden_layers(sat_mlp* m, const bf16* Z, int64_t R, bool training, cudaStream_t s) {
    cudaError_t e = gemm((int)R, m->h, m->n_in, Z, m->n_in, m->W1b, m->n_in, m->P + m->ob1, sat::EPI_GELU,
                         training ? m->pre1 : nullptr, m->h, 1.0f, nullptr, m->H1, m->h, training ? m->H1T : nullptr,
                         nullptr, m->cap, m->status, s);
    if (e != cudaSuccess) return e;
    return gemm((int)R, m->h, m->h, m->H1, m->h, m->W2b, m->h, m->P + m->ob2, sat::EPI_GELU,
                training ? m->pre2 : nullptr, m->h, 1.0f, nullptr, m->H2, m->h, training ? m->H2T : nullptr, nullptr,
                m->cap, m->status, s);
}

}  // namespace

// ----------------------------------------------------------------- C ABI --
extern "C" {

void sat_mlp_free(sat_mlp* m) {
    if (!m) return;
    for (void* a : m->allocs) cudaFree(a);
    delete m;
}

sat_status sat_mlp_create(uint32_t n_in, uint32_t n_hidden, uint32_t n_out, int64_t max_rows, uint64_t seed,
                          sat_mlp** out) {
    if (!out || n_in == 0 || n_hidden == 0 || n_out == 0 || max_rows <= 0 || (n_in % 8) || (n_hidden % 8))
        return sat::report_error(SAT_ERR_ARG, "bad MLP shape (n_in and n_hidden must be multiples of 8)");
    *out = nullptr;
    auto* m = new sat_mlp();
    cudaGetDevice(&m->device);
    m->n_in = (int)n_in;
    m->h = (int)n_hidden;
    m->n_out = (int)n_out;
    m->n_out_p = (int)((n_out + 7) / 8 * 8);
    m->cap = (max_rows + 7) / 8 * 8;
    m->oW1 = 0;
    m->ob1 = m->oW1 + (uint64_t)n_hidden * n_in;
    m->oW2 = m->ob1 + n_hidden;
    m->ob2 = m->oW2 + (uint64_t)n_hidden * n_hidden;
    m->oW3 = m->ob2 + n_hidden;
    m->ob3 = m->oW3 + (uint64_t)n_out * n_hidden;
    m->np = m->ob3 + n_out;
    auto alloc = [&](void** p, size_t bytes) {
        if (cudaMalloc(p, bytes < 16 ? 16 : bytes) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        m->allocs.push_back(*p);
        return true;
    };
    const size_t cap = (size_t)m->cap, h = n_hidden, no = n_out, nop = m->n_out_p;
    bool ok = alloc((void**)&m->P, m->np * 4) && alloc((void**)&m->G, m->np * 4) && alloc((void**)&m->M1, m->np * 4) &&
              alloc((void**)&m->M2, m->np * 4) && alloc((void**)&m->W1b, h * n_in * 2) &&
              alloc((void**)&m->W2b, h * h * 2) && alloc((void**)&m->W3b, no * h * 2) &&
              alloc((void**)&m->W2Tb, h * h * 2) && alloc((void**)&m->W3Tb, h * nop * 2) &&
              alloc((void**)&m->Z, cap * n_in * 2) && alloc((void**)&m->ZT, n_in * cap * 2) &&
              alloc((void**)&m->Zc, cap * n_in * 2) && alloc((void**)&m->pre1, cap * h * 4) &&
              alloc((void**)&m->pre2, cap * h * 4) && alloc((void**)&m->Y, cap * no * 4) &&
              alloc((void**)&m->H1, cap * h * 2) && alloc((void**)&m->H1T, h * cap * 2) &&
              alloc((void**)&m->H2, cap * h * 2) && alloc((void**)&m->H2T, h * cap * 2) &&
              alloc((void**)&m->dY, cap * nop * 2) && alloc((void**)&m->dYT, no * cap * 2) &&
              alloc((void**)&m->dA2, cap * h * 2) && alloc((void**)&m->dA2T, h * cap * 2) &&
              alloc((void**)&m->dA1, cap * h * 2) && alloc((void**)&m->dA1T, h * cap * 2) &&
              alloc((void**)&m->dist, cap * 4) && alloc((void**)&m->choice, cap * 4) &&
              alloc((void**)&m->loss_part, ((no + 31) / 32) * ((cap + 31) / 32) * 4 + 64) &&
              alloc((void**)&m->status, 4);
    if (!ok) {
        sat_mlp_free(m);
        return sat::report_error(SAT_ERR_OOM, "cudaMalloc failed for the MLP");
    }
    // PyTorch nn.Linear default init: U(-1/sqrt(fan_in), 1/sqrt(fan_in)), from SplitMix64.
    std::vector<float> host(m->np);
    uint64_t st = seed;
    auto next = [&]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    const uint64_t fan_in[6] = {n_in, n_in, n_hidden, n_hidden, n_hidden, n_hidden};
    const uint64_t off[7] = {m->oW1, m->ob1, m->oW2, m->ob2, m->oW3, m->ob3, m->np};
    for (int b = 0; b < 6; b++) {
        const double k = 1.0 / std::sqrt((double)fan_in[b]);
        for (uint64_t i = off[b]; i < off[b + 1]; i++) host[i] = (float)((2.0 * next() - 1.0) * k);
    }
    sat_status s = sat_mlp_set_params(m, host.data());
    if (s != SAT_OK) {
        sat_mlp_free(m);
        return s;
    }
    *out = m;
    return SAT_OK;
}

sat_status sat_mlp_num_params(const sat_mlp* m, uint64_t* n) {
    if (!m || !n) return sat::report_error(SAT_ERR_ARG, "NULL argument");
    *n = m->np;
    return SAT_OK;
}

sat_status sat_mlp_get_params(const sat_mlp* m, float* host) {
    if (!m || !host) return sat::report_error(SAT_ERR_ARG, "NULL argument");
    if (cudaMemcpy(host, m->P, m->np * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return sat::report_error(SAT_ERR_CUDA, "copy of MLP parameters failed");
    return SAT_OK;
}

sat_status sat_mlp_set_params(sat_mlp* m, const float* host) {
    if (!m || !host) return sat::report_error(SAT_ERR_ARG, "NULL argument");
    if (cudaMemcpy(m->P, host, m->np * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->M1, 0, m->np * 4) != cudaSuccess || cudaMemset(m->M2, 0, m->np * 4) != cudaSuccess ||
        cudaMemset(m->status, 0, 4) != cudaSuccess)
        return sat::report_error(SAT_ERR_CUDA, "upload of MLP parameters failed");
    m->t = 0;
    const int64_t nmax = std::max<int64_t>(std::max<int64_t>((int64_t)m->h * m->n_in, (int64_t)m->h * m->h),
                                           std::max<int64_t>((int64_t)m->n_out * m->h, (int64_t)m->h * m->n_out_p));
    refresh_kernel<<<blocks(nmax, 256), 256>>>(view_of(m));
    if (cudaDeviceSynchronize() != cudaSuccess) return sat::report_error(SAT_ERR_CUDA, "MLP weight refresh failed");
    return SAT_OK;
}

sat_status sat_mlp_draw_noise(sat_mlp* m, uint64_t seed, uint32_t round, void* z, int64_t rows, void* stream) {
    if (!m || (!z && rows > 0) || rows < 0) return sat::report_error(SAT_ERR_ARG, "bad argument");
    if (rows == 0) return SAT_OK;
    noise_kernel<<<std::min<unsigned>(blocks(rows * ((m->n_in + 3) / 4), 256), 148 * 16), 256, 0,
                   (cudaStream_t)stream>>>(
        seed, round, rows, m->n_in, (bf16*)z);
    if (cudaGetLastError() != cudaSuccess) return sat::report_error(SAT_ERR_CUDA, "noise launch failed");
    return SAT_OK;
}

sat_status sat_mlp_forward(sat_mlp* m, const void* z, int64_t rows, float tau, float* V, int64_t ldv, void* stream) {
    if (!m || !z || !V || rows < 0 || rows > m->cap || ldv < rows)
        return sat::report_error(SAT_ERR_ARG, "bad argument (rows must be <= the MLP's max_rows, ldv >= rows)");
    if (rows == 0) return SAT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = hidden_layers(m, (const bf16*)z, rows, false, s);
    if (e == cudaSuccess)
        e = gemm((int)rows, m->n_out, m->h, m->H2, m->h, m->W3b, m->h, m->P + m->ob3, sat::EPI_NONE, nullptr, 0, tau,
                 nullptr, nullptr, 0, nullptr, V, ldv, m->status, s);
    if (e != cudaSuccess) return sat::report_error(SAT_ERR_CUDA, std::string("MLP forward: ") + cudaGetErrorString(e));
    return SAT_OK;
}

sat_status sat_mlp_propose(sat_mlp* m, uint64_t seed, uint32_t round, float tau, float* V, int64_t ldv, int64_t B,
                           void* stream) {
    if (!m || B < 0 || B > m->cap) return sat::report_error(SAT_ERR_ARG, "batch exceeds the MLP's max_rows");
    sat_status st = sat_mlp_draw_noise(m, seed, round, m->Zc, B, stream);
    if (st != SAT_OK) return st;
    return sat_mlp_forward(m, m->Zc, B, tau, V, ldv, stream);
}

sat_status sat_mlp_imle_select(sat_mlp* m, const void* zc, const uint32_t* keys, int32_t key_words, int64_t S,
                               int32_t K, float* dist, int32_t* choice, void* stream) {
    if (!m || !zc || !keys || S < 0 || K < 1 || S * K > m->cap || key_words * 32 < m->n_out)
        return sat::report_error(SAT_ERR_ARG, "bad argument (S*K must be <= max_rows; keys must cover n_out bits)");
    if (S == 0) return SAT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t R = S * K;
    cudaError_t e = hidden_layers(m, (const bf16*)zc, R, false, s);
    if (e == cudaSuccess)
        e = gemm((int)R, m->n_out, m->h, m->H2, m->h, m->W3b, m->h, m->P + m->ob3, sat::EPI_NONE, nullptr, 0, 1.0f,
                 m->Y, nullptr, m->n_out, nullptr, nullptr, 0, m->status, s);
    if (e != cudaSuccess) return sat::report_error(SAT_ERR_CUDA, std::string("IMLE forward: ") + cudaGetErrorString(e));
    imle_dist_kernel<<<blocks(R * 32, 256), 256, 0, s>>>(m->Y, m->n_out, keys, key_words, K, R,
                                                         dist ? dist : m->dist);
    imle_choose_kernel<<<blocks(S, 128), 128, 0, s>>>(dist ? dist : m->dist, K, S, (const bf16*)zc, m->n_in, m->Z,
                                                      m->ZT, m->cap, choice ? choice : m->choice);
    if (cudaGetLastError() != cudaSuccess) return sat::report_error(SAT_ERR_CUDA, "IMLE launch failed");
    return SAT_OK;
}

// Loss and gradient at noise rows Z [S][n_in] (device bf16, or NULL = the rows
// chosen by the last sat_mlp_imle_select) against keys [S][key_words].
static sat_status loss_grad(sat_mlp* m, const bf16* z, const uint32_t* keys, int32_t kw, int64_t S, float* loss_host,
                            cudaStream_t s) {
    if (z) {
        if (cudaMemcpyAsync(m->Z, z, (size_t)S * m->n_in * 2, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return sat::report_error(SAT_ERR_CUDA, "copy of noise rows failed");
        transpose_z_kernel<<<blocks(S * m->n_in, 256), 256, 0, s>>>(m->Z, S, m->n_in, m->ZT, m->cap);
    }
    cudaError_t e = hidden_layers(m, m->Z, S, true, s);
    if (e == cudaSuccess)
        e = gemm((int)S, m->n_out, m->h, m->H2, m->h, m->W3b, m->h, m->P + m->ob3, sat::EPI_NONE, nullptr, 0, 1.0f,
                 m->Y, nullptr, m->n_out, nullptr, nullptr, 0, m->status, s);
    if (e != cudaSuccess) return sat::report_error(SAT_ERR_CUDA, std::string("MLP forward: ") + cudaGetErrorString(e));
    const float scale = 1.0f / ((float)S * (float)m->n_out);
    dim3 grid((unsigned)((m->n_out_p + 31) / 32), (unsigned)((S + 31) / 32));
    bce_grad_kernel<<<grid, 256, 0, s>>>(m->Y, m->n_out, m->n_out_p, keys, kw, S, scale, m->dY, m->dYT, m->cap,
                                         m->loss_part);
    // dW3 = dY^T H2, db3 = colsum(dY)
    e = gemm(m->n_out, m->h, (int)S, m->dYT, m->cap, m->H2T, m->cap, nullptr, sat::EPI_NONE, nullptr, 0, 1.0f,
             m->G + m->oW3, nullptr, m->h, nullptr, nullptr, 0, m->status, s);
    colsum_kernel<<<blocks(m->n_out, 128), 128, 0, s>>>(m->dY, S, m->n_out, m->n_out_p, m->G + m->ob3);
    // dA2 = (dY W3) * GELU'(pre2)
    if (e == cudaSuccess)
        e = gemm((int)S, m->h, m->n_out_p, m->dY, m->n_out_p, m->W3Tb, m->n_out_p, nullptr, sat::EPI_GELU_GRAD,
                 m->pre2, m->h, 1.0f, nullptr, m->dA2, m->h, m->dA2T, nullptr, m->cap, m->status, s);
    // dW2 = dA2^T H1, db2
    if (e == cudaSuccess)
        e = gemm(m->h, m->h, (int)S, m->dA2T, m->cap, m->H1T, m->cap, nullptr, sat::EPI_NONE, nullptr, 0, 1.0f,
                 m->G + m->oW2, nullptr, m->h, nullptr, nullptr, 0, m->status, s);
    colsum_kernel<<<blocks(m->h, 128), 128, 0, s>>>(m->dA2, S, m->h, m->h, m->G + m->ob2);
    // dA1 = (dA2 W2) * GELU'(pre1)
    if (e == cudaSuccess)
        e = gemm((int)S, m->h, m->h, m->dA2, m->h, m->W2Tb, m->h, nullptr, sat::EPI_GELU_GRAD, m->pre1, m->h, 1.0f,
                 nullptr, m->dA1, m->h, m->dA1T, nullptr, m->cap, m->status, s);
    // dW1 = dA1^T Z, db1
    if (e == cudaSuccess)
        e = gemm(m->h, m->n_in, (int)S, m->dA1T, m->cap, m->ZT, m->cap, nullptr, sat::EPI_NONE, nullptr, 0, 1.0f,
                 m->G + m->oW1, nullptr, m->n_in, nullptr, nullptr, 0, m->status, s);
    colsum_kernel<<<blocks(m->h, 128), 128, 0, s>>>(m->dA1, S, m->h, m->h, m->G + m->ob1);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return sat::report_error(SAT_ERR_CUDA, std::string("MLP backward: ") + cudaGetErrorString(e));
    if (loss_host) {
        const size_t np = (size_t)grid.x * grid.y;
        std::vector<float> part(np);
        if (cudaMemcpyAsync(part.data(), m->loss_part, np * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return sat::report_error(SAT_ERR_CUDA, "loss copy failed");
        double a = 0.0;
        for (float v : part) a += v;
        *loss_host = (float)(a / ((double)S * m->n_out));
    }
    return SAT_OK;
}

sat_status sat_mlp_loss_grad(sat_mlp* m, const void* z, const uint32_t* keys, int32_t key_words, int64_t S,
                             float* loss_host, float* grad_host, void* stream) {
    if (!m || !z || !keys || S <= 0 || S > m->cap || key_words * 32 < m->n_out)
        return sat::report_error(SAT_ERR_ARG, "bad argument (0 < S <= max_rows; keys must cover n_out bits)");
    cudaStream_t s = (cudaStream_t)stream;
    sat_status st = loss_grad(m, (const bf16*)z, keys, key_words, S, loss_host, s);
    if (st != SAT_OK) return st;
    if (grad_host) {
        if (cudaMemcpyAsync(grad_host, m->G, m->np * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return sat::report_error(SAT_ERR_CUDA, "gradient copy failed");
    }
    return SAT_OK;
}

// One Adam step of the master weights with gradient G (device [np]); then the BF16 copies.
static sat_status adam_apply(sat_mlp* m, const float* G, float lr, cudaStream_t s) {
    m->t++;
    // beta1, beta2 are the FP32 values 0.9f, 0.999f throughout: in the moment updates
    // (where 1 - beta is exact in FP32) and in the bias corrections (formed in FP64)
    const float b1 = 0.9f, b2 = 0.999f;
    const float step_size = (float)((double)lr / (1.0 - std::pow((double)b1, m->t)));
    const float bc2s = (float)std::sqrt(1.0 - std::pow((double)b2, m->t));
    adam_kernel<<<blocks((int64_t)m->np, 256), 256, 0, s>>>(m->P, G, m->M1, m->M2, m->np, lr, b1, b2, 1e-8f,
                                                            step_size, bc2s);
    const int64_t nmax = std::max<int64_t>(std::max<int64_t>((int64_t)m->h * m->n_in, (int64_t)m->h * m->h),
                                           std::max<int64_t>((int64_t)m->n_out * m->h, (int64_t)m->h * m->n_out_p));
    refresh_kernel<<<blocks(nmax, 256), 256, 0, s>>>(view_of(m));
    if (cudaGetLastError() != cudaSuccess) return sat::report_error(SAT_ERR_CUDA, "MLP update launch failed");
    return SAT_OK;
}

sat_status sat_mlp_apply_grad(sat_mlp* m, const float* grad, float lr, void* stream) {
    if (!m || !grad) return sat::report_error(SAT_ERR_ARG, "NULL argument");
    return adam_apply(m, grad, lr, (cudaStream_t)stream);
}

sat_status sat_mlp_train_step(sat_mlp* m, const uint32_t* keys, int32_t key_words, int64_t S, int32_t K, float lr,
                              uint64_t seed, uint32_t round, float* loss_host, void* stream) {
    if (!m || !keys || S <= 0 || K < 1 || S * K > m->cap || key_words * 32 < m->n_out)
        return sat::report_error(SAT_ERR_ARG, "bad argument (S*K must be <= max_rows)");
    cudaStream_t s = (cudaStream_t)stream;
    sat_status st = sat_mlp_draw_noise(m, seed, round, m->Zc, S * K, stream);
    if (st == SAT_OK) st = sat_mlp_imle_select(m, m->Zc, keys, key_words, S, K, nullptr, nullptr, stream);
    if (st == SAT_OK) st = loss_grad(m, nullptr, keys, key_words, S, loss_host, s);
    if (st != SAT_OK) return st;
    return adam_apply(m, m->G, lr, s);
}

sat_status sat_mlp_status(const sat_mlp* m, uint32_t* status) {
    if (!m || !status) return sat::report_error(SAT_ERR_ARG, "NULL argument");
    if (cudaMemcpy(status, m->status, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return sat::report_error(SAT_ERR_CUDA, "status copy failed");
    return SAT_OK;
}

}  // extern "C"
