// Instance-compiled round kernel (see compiled.cpp): limits, source generator and the
// per-plan compiled program.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

namespace sat {

struct Plan;

// Circuits the generator accepts: the live relaxed values of a step (the cone inputs' logits
// plus every cone node's activation) must fit the register file of one thread.
constexpr uint32_t ROUND_MAX_PI = 256;
constexpr uint64_t ROUND_MAX_LIVE = 224;     // n_cone_pi + n_cone
constexpr uint64_t ROUND_MAX_GATES = 4096;   // gates of the full circuit (Boolean pass)
constexpr size_t ROUND_MAX_LITERALS = 16384; // literals of the original clauses
constexpr int ROUND_THREADS = 128;
constexpr const char* ROUND_KERNEL_NAME = "sat_round_gd_kernel";

// Whether the plan's circuit is within the limits (why: the first limit it exceeds).
bool round_kernel_fits(const Plan& P, std::string* why);
// CUDA C++ source of the plan's round kernel (relax.cuh and philox.cuh are included by name).
std::string round_kernel_source(const Plan& P);

// NVRTC compilation of a round kernel's source to an sm_103a cubin; log = the compiler's
// messages (with verbose, ptxas's register and spill report).  False on failure.
// min_blocks: the minimum of resident blocks per SM asked of ptxas (__launch_bounds__).
bool compile_round_cubin(const std::string& source, bool verbose, std::vector<char>& cubin, std::string& log,
                         int min_blocks = 1);

// A compiled and loaded round kernel.  Libraries loaded with cudaLibraryLoadData are
// context-independent: one module serves every device of the process.
struct RoundModule {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
    int registers = 0, spill_bytes = 0, min_blocks = 1;
    double compile_ms = 0.0;
    ~RoundModule();
};

// A plan's round kernel: generated at plan creation, compiled and loaded on first use.
// Modules are shared through a process-wide cache keyed by the program text (the 32 most
// recently used are kept), so plans of the same circuit (sat_sample builds one per call)
// compile once.
struct CompiledRound {
    std::string source;
    std::mutex mu;
    bool tried = false;
    std::string error;
    std::shared_ptr<const RoundModule> mod;
    // Compile and load once (or take the cached module); later calls return the first
    // call's outcome.
    cudaError_t ensure(std::string& err);
    // One round for samples 0..B-1 (see sat_round_gd in the C ABI).
    cudaError_t launch(uint64_t seed, uint32_t round, float scale, float lr, int n_steps, float* V, int64_t ldv,
                       uint32_t* keys, uint32_t* valid, int64_t B, cudaStream_t s) const;
};

// Drops the cache's references (modules still held by plans stay loaded until those go).
void round_cache_clear();

}  // namespace sat
