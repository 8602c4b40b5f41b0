// sat_steps_noalloc: the fused optimisation steps of sat_steps, with the
// per-node scratch (activations and adjoints) taken from a fixed array in the
// library's own device memory instead of from the caller.
//
// Why it exists: some callers cannot allocate device memory at the point where
// they want to run the optimiser — for example a process whose whole device
// budget is handed to another allocator at start-up (a framework's caching
// pool, a serving loop with a fixed footprint), or a latency-critical loop
// that must not pay for cudaMalloc, which synchronises the device.  Those
// callers still pass V, m, v and loss, but need no act/adj buffers.
//
// The array below is a file-scope __device__ variable of SAT_NOALLOC_SCRATCH_BYTES:
// every GPU that loads this library holds it until the process exits.  Host
// code must not use its name as an address (on the host it is only a stand-in);
// the device address is looked up once per device with cudaGetSymbolAddress and
// kept for the life of the process (like every device object of the library, it
// does not survive a cudaDeviceReset).
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/satsampler.h"
#include "device.hpp"
#include "host.hpp"

struct sat_plan;  // defined in capi.cpp

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[SAT_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up on first use).
cudaError_t scratch_address(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_scratch_addr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" sat_status sat_steps_noalloc(const sat_plan* p, sat_act_dtype act_dtype, const sat_opt_params* o,
                                        float* V, float* m, float* v, int64_t ldv, float* loss, int32_t t0,
                                        int32_t n_steps, int64_t B, void* stream) {
    // the same argument checks as sat_steps, including that the plan lives on the current
    // device (the scratch address below is the current device's)
    sat_status st = sat::check_plan_call(p, B, ldv);
    if (st != SAT_OK) return st;
    const sat::DevPlan* dp = sat::plan_device(p);
    if (act_dtype < SAT_ACT_F32 || act_dtype > SAT_ACT_F16) return sat::report_error(SAT_ERR_ARG, "bad act_dtype");
    if (!sat::opt_params_ok(o) || t0 < 1 || n_steps < 0)
        return sat::report_error(SAT_ERR_ARG, "bad optimiser parameters or steps");
    if (B > 0 && dp->n_pi > 0 && (!V || (o->optimizer == SAT_OPT_ADAM && (!m || !v))))
        return sat::report_error(SAT_ERR_ARG, "NULL buffer");
    if (sat::steps_use_resident(*dp, (int)act_dtype)) {
        // the shared-memory resident kernel keeps activations and adjoints on chip: no scratch
        if (B == 0 || n_steps == 0) return SAT_OK;
        cudaError_t e = sat::launch_steps(*dp, dp->full, (int)act_dtype, sat::opt_params_of(o), V, m, v, ldv, nullptr, nullptr,
                                          loss, t0, n_steps, B, (cudaStream_t)stream);
        if (e != cudaSuccess) return sat::report_error(SAT_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
        return SAT_OK;
    }
    // the tiled kernel: act and adj blocks in the fixed array, each rounded up to 256 bytes
    const uint64_t tiles = (uint64_t)((B + SAT_TILE_SAMPLES - 1) / SAT_TILE_SAMPLES);
    const uint64_t act_elems = tiles * (uint64_t)dp->full.n_act_rows * SAT_TILE_SAMPLES;
    const uint64_t adj_elems = tiles * (uint64_t)dp->n_adj_rows * SAT_TILE_SAMPLES;
    const uint64_t act_bytes = (act_elems * (act_dtype == SAT_ACT_F32 ? 4u : 2u) + 255) / 256 * 256;
    const uint64_t adj_bytes = (adj_elems * 4u + 255) / 256 * 256;
    if (act_bytes + adj_bytes > SAT_NOALLOC_SCRATCH_BYTES)
        return sat::report_error(
            SAT_ERR_ARG, "sat_steps_noalloc needs " + std::to_string(act_bytes + adj_bytes) +
                             " bytes of scratch for this plan and batch; its fixed array holds " +
                             std::to_string((unsigned long long)SAT_NOALLOC_SCRATCH_BYTES) +
                             " bytes (use sat_steps with caller-provided buffers)");
    if (B == 0 || n_steps == 0) return SAT_OK;
    void* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess)
        return sat::report_error(SAT_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    unsigned char* s = static_cast<unsigned char*>(base);
    e = sat::launch_steps(*dp, dp->full, (int)act_dtype, sat::opt_params_of(o), V, m, v, ldv, s,
                          reinterpret_cast<float*>(s + act_bytes), loss, t0, n_steps, B, (cudaStream_t)stream);
    if (e != cudaSuccess) return sat::report_error(SAT_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return SAT_OK;
}
