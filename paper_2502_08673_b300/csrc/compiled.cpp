// Instance-compiled round kernel for small circuits: one sampling round of plain gradient
// descent (the paper's own setting, Section IV: GD on V for a few iterations) in one
// launch, with one thread per sample and every value in registers.
//
// The circuit is the kernel's code, not its data: the generator below writes the
// Philox/Box-Muller initialisation of every primary input (the draws of init_normal), the
// steps' forward (Eq. 5, the Table 1 bilinear forms), adjoint (Eq. 8 in gather form: each
// node sums its fan-out edges in CSR order, output seeds 2 (Y - T)) and GD update (Eq. 9),
// then the threshold bit of every input, the solution key, the Boolean pass over every
// gate and the check of the original clauses (Section II-A), both bitsliced over a warp's
// 32 samples with ballots.  Gate, edge, node and clause indices become register names and
// immediates; there are no index loads, no shared memory and no barriers.  The arithmetic
// is the separate kernels' own: the program embeds relax.cuh and philox.cuh verbatim and
// calls their functions (sigmoid, gate coefficients, gate evaluation, the input update,
// normal4), so keys, validity words and final logits are bit-identical to init_normal,
// the FP32 steps, threshold, Boolean pass and clause check run one after another.
//
// The program is compiled at run time with NVRTC for sm_103a (a cubin; nothing is JIT-
// compiled from PTX by the driver) and loaded with cudaLibraryLoadData.
#include <cuda_runtime.h>
#include <nvrtc.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <sstream>
#include <string>
#include <vector>

#include "compiled.hpp"
#include "host.hpp"
#include "jit_text.inc"  // kRelaxCuh, kPhiloxCuh: the text of relax.cuh and philox.cuh (written by the build)

namespace sat {
namespace {

// Headers that relax.cuh includes, reduced to what its device functions use.
const char* const kStubCudaRuntime = "#pragma once\n";
const char* const kStubCstdint =
    "#pragma once\n"
    "typedef signed char int8_t; typedef short int16_t; typedef int int32_t; typedef long long int64_t;\n"
    "typedef unsigned char uint8_t; typedef unsigned short uint16_t; typedef unsigned int uint32_t;\n"
    "typedef unsigned long long uint64_t;\n";
const char* const kStubDevice =
    "#pragma once\n"
    "namespace sat {\n"
    "struct OptParams {\n"
    "    int opt = 0;\n"
    "    float lr = 0.1f, b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;\n"
    "};\n"
    "}\n";

std::string fbits(float x) {
    char buf[32];
    uint32_t u;
    std::memcpy(&u, &x, 4);
    std::snprintf(buf, sizeof buf, "__int_as_float(0x%08xu)", u);
    return buf;
}

}  // namespace

bool round_kernel_fits(const Plan& P, std::string* why) {
    auto no = [&](const char* m) {
        if (why) *why = m;
        return false;
    };
    if (P.n_pi == 0) return no("no primary inputs");
    if (P.n_pi > ROUND_MAX_PI) return no("too many primary inputs");
    if (P.n_cone_pi + P.n_cone > ROUND_MAX_LIVE) return no("too many relaxed values to keep in registers");
    if (P.n_nodes - P.n_pi > ROUND_MAX_GATES) return no("too many gates");
    if (P.cl_node.size() > ROUND_MAX_LITERALS) return no("too many clause literals");
    return true;
}

std::string round_kernel_source(const Plan& P) {
    std::ostringstream s;
    const uint32_t npi = P.n_pi, ncpi = P.n_cone_pi;
    const int64_t ncone = (int64_t)P.n_cone;
    const int kw = (int)((npi + 31) / 32);
    std::vector<int64_t> cone_of_pi(npi, -1);
    for (uint32_t i = 0; i < ncpi; i++) cone_of_pi[P.cone_pi_row[i]] = i;

    s << "#include \"relax.cuh\"\n#include \"philox.cuh\"\n\n"
      << "#ifndef SAT_MIN_BLOCKS\n#define SAT_MIN_BLOCKS 1\n#endif\n"
      << "extern \"C\" __global__ void __launch_bounds__(" << ROUND_THREADS << ", SAT_MIN_BLOCKS) "
      << ROUND_KERNEL_NAME << "(\n"
      << "    unsigned long long seed, unsigned round, float scale, float lr, int n_steps, float* __restrict__ V,\n"
      << "    long long ldv, unsigned* __restrict__ keys, unsigned* __restrict__ valid, long long B) {\n"
      << "  const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;\n"
      << "  const unsigned lane = threadIdx.x & 31u, q = lane & 3u, quad = lane & ~3u;\n"
      << "  const bool in = b < B;\n"
      << "  const uint2 key = make_uint2((unsigned)seed, (unsigned)(seed >> 32));\n"
      << "  const unsigned grp = (unsigned)(b >> 2);\n";
    for (int g = 0; g < kw; g++) s << "  unsigned k" << g << " = 0u;\n";
    for (uint32_t i = 0; i < ncpi; i++) s << "  float v" << i << ";\n";

    // Initialisation, four input rows at a time: lane q of each quad draws the Philox block of
    // the group's q-th row for the quad's four samples (group b / 4), and the quad exchanges
    // the results so that every lane holds its own sample's value of the group's rows.  The
    // inputs outside every output's cone need only their threshold bits
    // (normal4_bits), after the cone inputs' initial logits (normal4).  When V is requested,
    // the host writes every input's initial logit with the init kernel before this launch.
    std::vector<uint32_t> cone_rows, free_rows;
    for (uint32_t r = 0; r < npi; r++) (cone_of_pi[r] >= 0 ? cone_rows : free_rows).push_back(r);
    auto row_select = [&](const std::vector<uint32_t>& rows, size_t g0) {
        std::ostringstream o;
        auto at = [&](size_t j) { return rows[std::min(g0 + j, rows.size() - 1)]; };
        o << "q == 0u ? " << at(0) << "u : q == 1u ? " << at(1) << "u : q == 2u ? " << at(2) << "u : " << at(3)
          << "u";
        return o.str();
    };
    s << "  // initial logits V = scale * z (the draws of init_normal)\n";
    for (size_t g0 = 0; g0 < cone_rows.size(); g0 += 4) {
        s << "  {\n    const float4 z = sat::normal4(grp, " << row_select(cone_rows, g0) << ", round, key);\n";
        for (size_t j = 0; j < 4 && g0 + j < cone_rows.size(); j++)
            s << "    {\n"
              << "      const float x0 = __shfl_sync(0xffffffffu, z.x, quad | " << j << "u);\n"
              << "      const float x1 = __shfl_sync(0xffffffffu, z.y, quad | " << j << "u);\n"
              << "      const float x2 = __shfl_sync(0xffffffffu, z.z, quad | " << j << "u);\n"
              << "      const float x3 = __shfl_sync(0xffffffffu, z.w, quad | " << j << "u);\n"
              << "      v" << cone_of_pi[cone_rows[g0 + j]]
              << " = scale * (q == 0u ? x0 : q == 1u ? x1 : q == 2u ? x2 : x3);\n"
              << "    }\n";
        s << "  }\n";
    }
    // their bits come from the signs alone unless the scale is so small that the products
    // could underflow
    auto free_bits = [&](const char* draw) {
        for (size_t g0 = 0; g0 < free_rows.size(); g0 += 4) {
            s << "    {\n      const unsigned nb = " << draw << "(grp, " << row_select(free_rows, g0)
              << ", round, key, " << (std::string(draw) == "sat::normal4_bits" ? "scale > 0.0f" : "scale") << ");\n";
            for (size_t j = 0; j < 4 && g0 + j < free_rows.size(); j++) {
                const uint32_t r = free_rows[g0 + j];
                s << "      k" << r / 32 << " |= ((__shfl_sync(0xffffffffu, nb, quad | " << j << "u) >> q) & 1u) << "
                  << r % 32 << ";\n";
            }
            s << "    }\n";
        }
    };
    if (!free_rows.empty()) {
        s << "  // threshold bits of the inputs outside every output's cone (fixed from here on)\n"
          << "  if (fabsf(scale) >= sat::BITS_MIN_SCALE) {\n";
        free_bits("sat::normal4_bits");
        s << "  } else {\n";
        free_bits("sat::normal4_bits_formed");
        s << "  }\n";
    }

    // The steps.
    s << "  #pragma unroll 1\n  for (int step = 0; step < n_steps; step++) {\n";
    for (uint32_t i = 0; i < ncpi; i++) s << "    const float a" << i << " = sat::sigmoidf_(v" << i << ");\n";
    for (int64_t n = ncpi; n < ncone; n++) {
        const size_t g = (size_t)(n - ncpi);
        s << "    const float a" << n << " = sat::gate_apply(sat::gate_coeffs(" << (unsigned)P.c_gop[g] << "u), a"
          << P.c_in0[g] << ", a" << P.c_in1[g] << ");\n";
    }
    // adjoints, levels from the top down (a node's consumers lie above it)
    const int32_t nlev = (int32_t)P.c_level_off.size() - 2;
    for (int32_t l = nlev; l >= 0; l--) {
        const int64_t lo = l == 0 ? 0 : P.c_level_off[l], hi = l == 0 ? ncpi : P.c_level_off[l + 1];
        for (int64_t u = lo; u < hi; u++) {
            s << "    float d" << u << " = 0.0f;\n";
            for (int64_t e = P.fo_off[u]; e < P.fo_off[u + 1]; e++) {
                const std::string ga = P.fo_g[e] < 0 ? std::string("1.0f") : "d" + std::to_string(P.fo_g[e]);
                s << "    d" << u << " = fmaf(" << ga << ", fmaf(" << fbits((float)P.fo_c1[e]) << ", a" << P.fo_sib[e]
                  << ", " << fbits((float)P.fo_c0[e]) << "), d" << u << ");\n";
            }
        }
    }
    // GD on the cone inputs (Eq. 9), through the same update routine
    for (uint32_t i = 0; i < ncpi; i++)
        s << "    { sat::OptParams o; o.opt = 1; o.lr = lr; float nv = 0.0f;\n"
          << "      sat::input_update_p<true>(o, &nv, nullptr, nullptr, nullptr, 0, v" << i << ", a" << i << ", d" << i
          << ", 0.0f, 0.0f, 1.0f, 1.0f); v" << i << " = nv; }\n";
    s << "  }\n";

    // Threshold and key of the cone inputs; final logits.
    for (uint32_t i = 0; i < ncpi; i++) {
        const int32_t r = P.cone_pi_row[i];
        s << "  k" << r / 32 << " |= (v" << i << " > 0.0f ? 1u : 0u) << " << r % 32 << ";\n"
          << "  if (V != nullptr && in) V[" << r << "LL * ldv + b] = v" << i << ";\n";
    }
    s << "  if (in) {\n";
    for (int g = 0; g < kw; g++) s << "    keys[b * " << kw << "LL + " << g << "] = k" << g << ";\n";
    s << "  }\n";

    // Boolean pass and clause check, 32 samples per word (lane j: sample 32 (b / 32) + j).
    s << "  // bitsliced Boolean pass over every gate\n";
    for (uint32_t r = 0; r < npi; r++)
        s << "  const unsigned w" << r << " = __ballot_sync(0xffffffffu, (k" << r / 32 << " >> " << r % 32
          << ") & 1u);\n";
    for (size_t g = 0; g < P.in0.size(); g++) {
        const unsigned gop = P.gop[g];
        const std::string a = std::string((gop & 4) ? "~w" : "w") + std::to_string(P.in0[g]);
        const std::string bb = std::string((gop & 8) ? "~w" : "w") + std::to_string(P.in1[g]);
        const char* op = (gop & 3) == 0 ? " & " : (gop & 3) == 1 ? " | " : " ^ ";
        s << "  const unsigned w" << (uint64_t)P.n_pi + g << " = " << a << op << bb << ";\n";
    }
    s << "  // the original clauses\n  unsigned ok = 0xffffffffu;\n";
    for (size_t c = 0; c + 1 < P.cl_off.size(); c++) {
        s << "  ok &= ";
        for (int64_t i = P.cl_off[c]; i < P.cl_off[c + 1]; i++)
            s << (i > P.cl_off[c] ? " | " : "") << (P.cl_neg[i] ? "~w" : "w") << P.cl_node[i];
        if (P.cl_off[c + 1] == P.cl_off[c]) s << "0u";
        s << ";\n";
    }
    s << "  const unsigned live = __ballot_sync(0xffffffffu, in);\n"
      << "  if (lane == 0u && in) valid[b >> 5] = ok & live;\n"
      << "}\n";
    return s.str();
}

RoundModule::~RoundModule() {
    if (lib) cudaLibraryUnload(lib);
}

bool compile_round_cubin(const std::string& source, bool verbose, std::vector<char>& cubin, std::string& log,
                         int min_blocks) {
    nvrtcProgram prog = nullptr;
    const char* headers[] = {kRelaxCuh, kPhiloxCuh, kStubCudaRuntime, kStubCstdint, kStubDevice};
    const char* names[] = {"relax.cuh", "philox.cuh", "cuda_runtime.h", "cstdint", "device.hpp"};
    if (nvrtcCreateProgram(&prog, source.c_str(), "sat_round.cu", 5, headers, names) != NVRTC_SUCCESS) {
        log = "nvrtcCreateProgram failed";
        return false;
    }
    // IEEE division and square root, fma contraction on, no flush to zero: nvcc's defaults,
    // which the separate kernels are built with
    const std::string mb = "-DSAT_MIN_BLOCKS=" + std::to_string(min_blocks);
    const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "--fmad=true", "--prec-div=true",
                          "--prec-sqrt=true", "--ftz=false", mb.c_str(), "--ptxas-options=-v"};
    const nvrtcResult rc = nvrtcCompileProgram(prog, verbose ? 8 : 7, opts);
    size_t log_size = 0;
    nvrtcGetProgramLogSize(prog, &log_size);
    log.assign(log_size, '\0');
    if (log_size > 1) nvrtcGetProgramLog(prog, &log[0]);
    while (!log.empty() && log.back() == '\0') log.pop_back();
    if (rc != NVRTC_SUCCESS) {
        log = std::string("NVRTC compilation failed: ") + nvrtcGetErrorString(rc) + "\n" + log;
        nvrtcDestroyProgram(&prog);
        return false;
    }
    size_t cubin_size = 0;
    nvrtcGetCUBINSize(prog, &cubin_size);
    cubin.resize(cubin_size);
    nvrtcGetCUBIN(prog, cubin.data());
    nvrtcDestroyProgram(&prog);
    return true;
}

namespace {
constexpr size_t ROUND_CACHE_ENTRIES = 32;
std::mutex g_cache_mu;
std::vector<std::pair<std::string, std::shared_ptr<const RoundModule>>> g_cache;  // most recent last

std::shared_ptr<const RoundModule> cache_find(const std::string& source) {
    for (size_t i = 0; i < g_cache.size(); i++)
        if (g_cache[i].first == source) {
            auto e = std::move(g_cache[i]);
            g_cache.erase(g_cache.begin() + (long)i);
            g_cache.push_back(std::move(e));
            return g_cache.back().second;
        }
    return nullptr;
}
}  // namespace

void round_cache_clear() {
    std::lock_guard<std::mutex> g(g_cache_mu);
    g_cache.clear();
}

namespace {
// Compiles and loads the program with the given minimum of resident blocks per SM
// (__launch_bounds__), or returns null with err set.
std::shared_ptr<RoundModule> build_module(const std::string& source, int min_blocks, std::string& err) {
    std::vector<char> cubin;
    std::string log;
    if (!compile_round_cubin(source, false, cubin, log, min_blocks)) {
        err = log;
        return nullptr;
    }
    auto m = std::make_shared<RoundModule>();
    cudaError_t e = cudaLibraryLoadData(&m->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&m->kern, m->lib, ROUND_KERNEL_NAME);
    cudaFuncAttributes fa{};
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(m->kern));
    if (e != cudaSuccess) {
        err = std::string("loading the compiled round kernel failed: ") + cudaGetErrorString(e);
        return nullptr;
    }
    m->registers = fa.numRegs;
    m->spill_bytes = (int)fa.localSizeBytes;
    m->min_blocks = min_blocks;
    return m;
}

// Blocks of ROUND_THREADS threads that the register file holds (registers are allocated
// per warp in units of 256, i.e. 8 per thread).
int blocks_per_sm(int registers) {
    const int per_thread = (std::max(registers, 1) + 7) / 8 * 8;
    return std::min(65536 / (per_thread * ROUND_THREADS), 2048 / ROUND_THREADS);
}
}  // namespace

cudaError_t CompiledRound::ensure(std::string& err) {
    std::lock_guard<std::mutex> g(mu);
    if (tried) {
        err = error;
        return mod ? cudaSuccess : cudaErrorInvalidValue;
    }
    tried = true;
    // one compilation per program text at a time: the cache lock is held across it
    std::lock_guard<std::mutex> cg(g_cache_mu);
    if ((mod = cache_find(source))) {
        err.clear();
        return cudaSuccess;
    }
    const auto t0 = std::chrono::steady_clock::now();
    std::shared_ptr<RoundModule> m = build_module(source, 1, error);
    if (!m) {
        err = error;
        return cudaErrorInvalidValue;
    }
    // More resident warps hide more of the kernel's dependency latency (paper setting: 79
    // registers and 6 blocks per SM, 0.244 ms, against 89 and 5 blocks, 0.258 ms): ask
    // ptxas for one more block per SM while that keeps every value in registers (at most
    // two more compilations).
    for (int tries = 0; tries < 2 && m->spill_bytes == 0; tries++) {
        const int want = blocks_per_sm(m->registers) + 1;
        if (want > 2048 / ROUND_THREADS) break;
        std::string e2;
        std::shared_ptr<RoundModule> t = build_module(source, want, e2);
        if (!t || t->spill_bytes != 0 || blocks_per_sm(t->registers) < want) break;
        m = t;
    }
    m->compile_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    mod = m;
    g_cache.emplace_back(source, m);
    if (g_cache.size() > ROUND_CACHE_ENTRIES) g_cache.erase(g_cache.begin());
    err.clear();
    return cudaSuccess;
}

cudaError_t CompiledRound::launch(uint64_t seed, uint32_t round, float scale, float lr, int n_steps, float* V,
                                  int64_t ldv, uint32_t* keys, uint32_t* valid, int64_t B, cudaStream_t s) const {
    if (!mod) return cudaErrorInvalidValue;
    if (B == 0) return cudaSuccess;
    unsigned long long a_seed = seed;
    unsigned a_round = round;
    float a_scale = scale, a_lr = lr;
    int a_steps = n_steps;
    long long a_ldv = ldv, a_B = B;
    void* args[] = {&a_seed, &a_round, &a_scale, &a_lr, &a_steps, &V, &a_ldv, &keys, &valid, &a_B};
    const unsigned grid = (unsigned)((B + ROUND_THREADS - 1) / ROUND_THREADS);
    return cudaLaunchKernel(reinterpret_cast<const void*>(mod->kern), dim3(grid), dim3(ROUND_THREADS), args, 0, s);
}

}  // namespace sat
