// Canonical order of the distinct solutions on the device: the dedup keys sorted
// ascending by their top 64 bits (the highest word most significant), ties by pool
// index, with a bitonic network (Batcher 1968) over (prefix, index) pairs padded to a
// power of two; then the keys are gathered in that order.  Keys whose prefixes tie
// (possible only with more than 64 key bits) are put in full-key order on the host.
#include <cuda_runtime.h>

#include <cstdint>

#include "device.hpp"

namespace sat {
namespace {

constexpr int SORT_BLOCK = 2048;  // elements per shared-memory block (1024 threads, one pair each)

__device__ __forceinline__ bool pair_greater(uint64_t ha, uint32_t ia, uint64_t hb, uint32_t ib) {
    return ha > hb || (ha == hb && ia > ib);
}

// (prefix, index) of pool entry i; entries past n are padding that sorts last.
__global__ void key_prefix_kernel(const uint32_t* keys, int kw, uint64_t n, uint64_t n2, uint64_t* hi,
                                  uint32_t* idx) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (uint64_t)gridDim.x * blockDim.x) {
        if (i < n) {
            const uint32_t* k = keys + i * (uint64_t)kw;
            uint64_t h = (uint64_t)k[kw - 1] << 32;
            if (kw >= 2) h |= k[kw - 2];
            hi[i] = h;
            idx[i] = (uint32_t)i;
        } else {
            hi[i] = ~0ull;
            idx[i] = 0xFFFFFFFFu;
        }
    }
}

// One (k, j) stage of the network whose pairs (i, i + j) span more than a shared-memory
// block: compare-exchange, ascending where (i & k) == 0.
__global__ void bitonic_global_kernel(uint64_t* hi, uint32_t* idx, uint64_t n2, uint64_t k, uint64_t j) {
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n2 / 2; p += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = (p / j) * 2 * j + (p % j), l = i + j;
        const bool up = (i & k) == 0;
        const uint64_t ha = hi[i], hb = hi[l];
        const uint32_t ia = idx[i], ib = idx[l];
        if (pair_greater(ha, ia, hb, ib) == up) {
            hi[i] = hb;
            hi[l] = ha;
            idx[i] = ib;
            idx[l] = ia;
        }
    }
}

// All stages with j < block size for the k values in [k_lo, k_hi] (doubling), inside one
// block of min(n2, SORT_BLOCK) elements in shared memory.
__global__ void __launch_bounds__(SORT_BLOCK / 2) bitonic_shared_kernel(uint64_t* hi, uint32_t* idx, uint64_t n2,
                                                                         uint64_t k_lo, uint64_t k_hi) {
    __shared__ uint64_t sh[SORT_BLOCK];
    __shared__ uint32_t si[SORT_BLOCK];
    const uint64_t m = n2 < (uint64_t)SORT_BLOCK ? n2 : (uint64_t)SORT_BLOCK;
    const uint64_t base = (uint64_t)blockIdx.x * m;
    for (uint64_t t = threadIdx.x; t < m; t += blockDim.x) {
        sh[t] = hi[base + t];
        si[t] = idx[base + t];
    }
    __syncthreads();
    for (uint64_t k = k_lo; k <= k_hi; k *= 2) {
        for (uint64_t j = (k / 2 < m / 2 ? k / 2 : m / 2); j >= 1; j /= 2) {
            for (uint64_t p = threadIdx.x; p < m / 2; p += blockDim.x) {
                const uint64_t i = (p / j) * 2 * j + (p % j), l = i + j;
                const bool up = ((base + i) & k) == 0;
                const uint64_t ha = sh[i], hb = sh[l];
                const uint32_t ia = si[i], ib = si[l];
                if (pair_greater(ha, ia, hb, ib) == up) {
                    sh[i] = hb;
                    sh[l] = ha;
                    si[i] = ib;
                    si[l] = ia;
                }
            }
            __syncthreads();
        }
    }
    for (uint64_t t = threadIdx.x; t < m; t += blockDim.x) {
        hi[base + t] = sh[t];
        idx[base + t] = si[t];
    }
}

__global__ void gather_keys_kernel(const uint32_t* keys, int kw, uint64_t n, const uint32_t* idx, uint32_t* out) {
    const uint64_t total = n * (uint64_t)kw;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r = e / (uint64_t)kw, w = e % (uint64_t)kw;
        out[e] = keys[(uint64_t)idx[r] * kw + w];
    }
}

unsigned grid_for(uint64_t work, unsigned block) {
    const uint64_t g = (work + block - 1) / block;
    return (unsigned)(g < 148ull * 32 ? (g ? g : 1) : 148ull * 32);
}

}  // namespace

uint64_t key_order_pad(uint64_t n) {
    uint64_t n2 = 1;
    while (n2 < n) n2 <<= 1;
    return n2;
}

cudaError_t launch_key_order(const uint32_t* keys, int kw, uint64_t n, uint64_t* hi, uint32_t* idx, uint32_t* out,
                             cudaStream_t s) {
    if (n == 0 || kw <= 0) return cudaSuccess;
    const uint64_t n2 = key_order_pad(n);
    key_prefix_kernel<<<grid_for(n2, 256), 256, 0, s>>>(keys, kw, n, n2, hi, idx);
    const uint64_t m = n2 < (uint64_t)SORT_BLOCK ? n2 : (uint64_t)SORT_BLOCK;
    const unsigned blocks = (unsigned)(n2 / m);
    // every k up to the block size inside shared memory
    bitonic_shared_kernel<<<blocks, SORT_BLOCK / 2, 0, s>>>(hi, idx, n2, 2, m);
    for (uint64_t k = 2 * m; k <= n2; k *= 2) {
        for (uint64_t j = k / 2; j >= m; j /= 2) bitonic_global_kernel<<<grid_for(n2 / 2, 256), 256, 0, s>>>(hi, idx, n2, k, j);
        bitonic_shared_kernel<<<blocks, SORT_BLOCK / 2, 0, s>>>(hi, idx, n2, k, k);
    }
    gather_keys_kernel<<<grid_for(n * (uint64_t)kw, 256), 256, 0, s>>>(keys, kw, n, idx, out);
    return cudaGetLastError();
}

}  // namespace sat
