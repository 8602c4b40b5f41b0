// extern "C" boundary of the sampler library: argument checks, object
// lifetimes, device uploads and the end-to-end round loop.  Every step of the
// path runs in the kernels of steps.cu, resident.cu and sample.cu.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstdint>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <utility>
#include <vector>

#include "../../include/satsampler.h"
#include "compiled.hpp"
#include "device.hpp"
#include "host.hpp"

static_assert(SAT_TILE == SAT_TILE_SAMPLES, "ABI tile width");
static_assert((int)SAT_STEP_KERNEL_AUTO == (int)sat::STEP_KERNEL_AUTO &&
                  (int)SAT_STEP_KERNEL_TILED == (int)sat::STEP_KERNEL_TILED &&
                  (int)SAT_STEP_KERNEL_RESIDENT == (int)sat::STEP_KERNEL_RESIDENT,
              "ABI step kernel codes");

struct sat_cnf {
    sat::Cnf cnf;
};

struct sat_circuit {
    sat::Circuit circ;
    sat::Plan plan;
    double plan_ms = 0.0;
    uint64_t cnf_clauses = 0;
};

struct sat_plan {
    int device = 0;
    sat::DevPlan dp;
    std::vector<void*> allocs;
    std::vector<int32_t> h_c_level_off, h_f_level_off;
    // host copies of the cone records (full layout), for building recomputation layouts
    std::vector<int2> h_gate;
    std::vector<int4> h_edge;
    std::vector<int32_t> h_out;
    // recomputation layouts, built on first use (segment length -> layout)
    mutable std::mutex lay_mu;
    mutable std::map<int32_t, sat::DevAct> layouts;
    mutable std::vector<void*> lay_allocs;
    std::vector<uint32_t> pi_var;
    std::vector<int64_t> var_cone, var_full;
    std::vector<uint8_t> var_neg;
    // host copy of the full schedule, for expanding solution keys
    std::vector<int32_t> f_in0, f_in1;
    std::vector<uint8_t> f_gop;
    sat_plan_info info{};
    // the instance-compiled round kernel (circuits within its limits), compiled on first use
    std::unique_ptr<sat::CompiledRound> round;
};

struct sat_dedup {
    int device = 0;
    sat::DevDedup d;
    int64_t max_batch = 0;
    unsigned long long* slot_of = nullptr;
};

// Allocator whose value-initialisation leaves elements uninitialised: the key buffer is
// written in full by the download, so resizing it need not zero it first.
template <typename T>
struct uninit_allocator : std::allocator<T> {
    template <typename U>
    struct rebind {
        using other = uninit_allocator<U>;
    };
    uninit_allocator() = default;
    template <typename U>
    uninit_allocator(const uninit_allocator<U>&) noexcept {}
    template <typename U>
    void construct(U* p) noexcept {
        ::new ((void*)p) U;
    }
    template <typename U, typename... A>
    void construct(U* p, A&&... a) {
        ::new ((void*)p) U(std::forward<A>(a)...);
    }
};

using KeyBuffer = std::vector<uint32_t, uninit_allocator<uint32_t>>;

struct sat_solutions {
    uint32_t n_vars = 0, n_pi = 0, key_words = 0;
    uint64_t count = 0;
    KeyBuffer keys;                    // [count][key_words], canonical order
    std::vector<int32_t> f_in0, f_in1;
    std::vector<uint8_t> f_gop;
    std::vector<int64_t> var_full;
    std::vector<uint8_t> var_neg;
};

namespace {

thread_local std::string g_err;

sat_status fail(sat_status s, const std::string& m) {
    g_err = m;
    return s;
}

#define CK(expr)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (expr);                                                                  \
        if (e_ != cudaSuccess) return fail(SAT_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// The library's own stream-ordered memory pool of each device.  It keeps the memory it
// has reserved when buffers are freed (release threshold: unlimited), so a repeated
// call maps no new device memory and freeing does not synchronise the device;
// sat_release_cached_memory hands the reserve back.
constexpr int MAX_DEVICES = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[MAX_DEVICES] = {};

cudaError_t library_pool(cudaMemPool_t* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return e;
        uint64_t keep = ~0ull;
        if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        g_pools[dev] = pool;
    }
    *out = g_pools[dev];
    return cudaSuccess;
}

// Device arrays of plans and dedup sets: from the library pool, in stream order on the
// legacy default stream (ordered after the work of every blocking stream), so that
// creating and freeing the objects of an end-to-end call neither maps memory nor waits
// for the device.  An allocation the pool cannot serve is retried once after the pool's
// idle reserve is returned.
bool obj_alloc(void** p, size_t n) {
    cudaMemPool_t pool = nullptr;
    if (library_pool(&pool) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (cudaMallocFromPoolAsync(p, n ? n : 16, pool, 0) == cudaSuccess) return true;
    cudaGetLastError();
    cudaMemPoolTrimTo(pool, 0);
    if (cudaMallocFromPoolAsync(p, n ? n : 16, pool, 0) == cudaSuccess) return true;
    cudaGetLastError();
    *p = nullptr;
    return false;
}
void obj_free(void* p) {
    if (p) cudaFreeAsync(p, 0);
}

template <typename T>
sat_status upload_to(std::vector<void*>& allocs, const std::vector<T>& h, const T** dst) {
    *dst = nullptr;
    if (h.empty()) return SAT_OK;
    void* d = nullptr;
    if (!obj_alloc(&d, h.size() * sizeof(T))) return fail(SAT_ERR_OOM, "device allocation failed for plan array");
    allocs.push_back(d);
    CK(cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    *dst = (const T*)d;
    return SAT_OK;
}
template <typename T>
sat_status upload(sat_plan* p, const std::vector<T>& h, const T** dst) {
    p->info.upload_bytes += h.size() * sizeof(T);
    return upload_to(p->allocs, h, dst);
}

// Every row a step kernel gathers or stores through these records must lie inside its
// tile's block: checked once on the host, so that the kernels need no per-access bounds
// test (a TMA gather outside the tensor map would read fill values, a store would not).
bool records_in_range(const std::vector<int2>& gate, const std::vector<int4>& edge,
                             const std::vector<int32_t>& out_row, int64_t act_rows, int64_t adj_rows) {
    auto ok = [](int64_t r, int64_t n) { return r >= 0 && r < n; };
    for (const int2& g : gate)
        if (!ok(g.x & 0x0FFFFFFF, act_rows) || !ok(g.y, act_rows)) return false;
    for (const int4& e : edge)
        if ((e.x != -1 && !ok(e.x, adj_rows)) || !ok(e.y & 0x7FFFFFFF, act_rows)) return false;
    for (int32_t r : out_row)
        if (!ok(r, act_rows)) return false;
    return true;
}

sat_status check_device(int device) {
    int cur = -1;
    CK(cudaGetDevice(&cur));
    if (cur != device) return fail(SAT_ERR_ARG, "object belongs to another device than the current one");
    return SAT_OK;
}

int64_t round32(int64_t x) { return (x + 31) / 32 * 32; }

sat_status check_layout(const sat_plan* p, int64_t B, int64_t ldv) {
    if (!p) return fail(SAT_ERR_ARG, "plan is NULL");
    if (B < 0) return fail(SAT_ERR_ARG, "B < 0");
    if (ldv >= 0 && ldv < B) return fail(SAT_ERR_ARG, "ldv < B");
    if (B >= (1ll << 31)) return fail(SAT_ERR_ARG, "B must be < 2^31");
    return check_device(p->device);
}

cudaStream_t S(void* s) { return (cudaStream_t)s; }

sat::OptParams opt_of(const sat_opt_params* o) {
    sat::OptParams r;
    r.opt = o->optimizer;
    r.lr = o->lr;
    r.b1 = o->beta1;
    r.b2 = o->beta2;
    r.eps = o->eps;
    return r;
}

bool opt_ok(const sat_opt_params* o) {
    return o && (o->optimizer == SAT_OPT_ADAM || o->optimizer == SAT_OPT_GD) &&
           (o->optimizer == SAT_OPT_GD || (o->beta1 >= 0 && o->beta1 < 1 && o->beta2 >= 0 && o->beta2 < 1));
}

}  // namespace

namespace sat {
sat_status report_error(sat_status s, const std::string& msg) { return fail(s, msg); }
const DevPlan* plan_device(const sat_plan* p) { return &p->dp; }
sat_status check_plan_call(const sat_plan* p, int64_t B, int64_t ldv) { return check_layout(p, B, ldv); }
bool opt_params_ok(const sat_opt_params* o) { return opt_ok(o); }
OptParams opt_params_of(const sat_opt_params* o) { return opt_of(o); }
}  // namespace sat

namespace sat {
// sample.cu: the angle-grid sign check behind sat_diag_angle_signs
cudaError_t launch_angle_signs_diag(unsigned* mismatches, cudaStream_t s);
}  // namespace sat

extern "C" {

const char* sat_version(void) { return "satsampler 0.1 (sm_103a)"; }
const char* sat_last_error(void) { return g_err.c_str(); }

// ------------------------------------------------------------------ CNF --
sat_status sat_cnf_from_dimacs(const char* buf, size_t len, sat_cnf** out) {
    if (!out || (!buf && len)) return fail(SAT_ERR_ARG, "NULL argument");
    *out = nullptr;
    try {
        std::string copy(buf ? buf : "", len);
        auto* c = new sat_cnf();
        std::string err;
        if (!sat::parse_dimacs(copy.c_str(), copy.size(), c->cnf, err)) {
            delete c;
            return fail(SAT_ERR_PARSE, err);
        }
        *out = c;
        return SAT_OK;
    } catch (const std::bad_alloc&) {
        return fail(SAT_ERR_OOM, "host allocation failed");
    }
}

sat_status sat_cnf_from_file(const char* path, sat_cnf** out) {
    if (!path || !out) return fail(SAT_ERR_ARG, "NULL argument");
    std::ifstream f(path, std::ios::binary);
    if (!f) return fail(SAT_ERR_ARG, std::string("cannot open ") + path);
    std::stringstream ss;
    ss << f.rdbuf();
    std::string s = ss.str();
    return sat_cnf_from_dimacs(s.data(), s.size(), out);
}

sat_status sat_cnf_info(const sat_cnf* c, uint32_t* n_vars, uint64_t* n_clauses, uint64_t* n_lits) {
    if (!c) return fail(SAT_ERR_ARG, "NULL cnf");
    if (n_vars) *n_vars = c->cnf.n_vars;
    if (n_clauses) *n_clauses = c->cnf.n_clauses();
    if (n_lits) *n_lits = c->cnf.lits.size();
    return SAT_OK;
}

void sat_cnf_free(sat_cnf* c) { delete c; }

// ------------------------------------------------------- transformation --
sat_status sat_circuit_build(const sat_cnf* cnf, const sat_build_opts* opts, sat_circuit** out,
                             sat_build_stats* st) {
    if (!cnf || !out) return fail(SAT_ERR_ARG, "NULL argument");
    *out = nullptr;
    sat::TransformOpts to;
    if (opts) {
        to.max_support = opts->max_support;
        to.max_window = opts->max_window;
        to.direct = opts->direct != 0;
        to.reorder = opts->reorder != 0;
    }
    try {
        auto* c = new sat_circuit();
        std::string err;
        if (!sat::transform(cnf->cnf, to, c->circ, err)) {
            delete c;
            return fail(err.rfind("empty clause", 0) == 0 ? SAT_ERR_UNSAT_TRIVIAL : SAT_ERR_ARG, err);
        }
        auto t0 = std::chrono::steady_clock::now();
        if (!sat::build_plan(c->circ, cnf->cnf, c->plan, err)) {
            delete c;
            return fail(SAT_ERR_ARG, err);
        }
        c->plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        c->cnf_clauses = cnf->cnf.n_clauses();
        if (st) {
            const sat::Plan& P = c->plan;
            *st = sat_build_stats{};
            st->n_vars = c->circ.n_vars;
            st->n_pi = (uint32_t)c->circ.pis.size();
            st->n_iv = (uint32_t)c->circ.defs.size();
            st->n_outputs = (uint32_t)c->circ.outputs.size();
            st->n_const = c->circ.n_const;
            st->n_gates = P.in0.size();
            st->n_cone_pi = P.n_cone_pi;
            st->n_cone_gates = P.c_in0.size();
            st->n_levels = (uint32_t)(P.level_off.size() - 2);
            st->n_cone_levels = (uint32_t)(P.c_level_off.size() - 2);
            st->max_span = P.max_span;
            st->ops_cnf = P.ops_cnf;
            st->ops_circuit = P.ops_circuit;
            st->transform_ms = c->circ.wall_ms;
            st->plan_ms = c->plan_ms;
        }
        *out = c;
        return SAT_OK;
    } catch (const std::bad_alloc&) {
        return fail(SAT_ERR_OOM, "host allocation failed");
    }
}

sat_status sat_circuit_dump(const sat_circuit* c, char* buf, size_t cap, size_t* len) {
    if (!c) return fail(SAT_ERR_ARG, "NULL circuit");
    std::string s = sat::circuit_dump(c->circ);
    if (len) *len = s.size();
    if (buf && cap) {
        size_t n = std::min(cap, s.size() + 1);
        std::memcpy(buf, s.c_str(), n);
    }
    return SAT_OK;
}

sat_status sat_circuit_round_program(const sat_circuit* c, int32_t compile, char* buf, size_t cap, size_t* len) {
    if (!c) return fail(SAT_ERR_ARG, "NULL circuit");
    std::string why;
    if (!sat::round_kernel_fits(c->plan, &why)) return fail(SAT_ERR_ARG, "no compiled round kernel: " + why);
    std::string text = sat::round_kernel_source(c->plan);
    bool ok = true;
    if (compile) {
        std::vector<char> cubin;
        ok = sat::compile_round_cubin(text, true, cubin, text);
    }
    if (len) *len = text.size();
    if (buf && cap) {
        size_t n = std::min(cap, text.size() + 1);
        std::memcpy(buf, text.c_str(), n);
    }
    return ok ? SAT_OK : fail(SAT_ERR_CUDA, text);
}

void sat_circuit_free(sat_circuit* c) { delete c; }

// ---------------------------------------------------------------- plan --
sat_status sat_plan_set_step_kernel(sat_plan* p, int32_t kind) {
    if (!p) return fail(SAT_ERR_ARG, "NULL plan");
    if (kind < SAT_STEP_KERNEL_AUTO || kind > SAT_STEP_KERNEL_RESIDENT) return fail(SAT_ERR_ARG, "bad step kernel");
    if (kind == SAT_STEP_KERNEL_RESIDENT && !sat::resident_config(p->dp, sat::ACT_BF16, nullptr, nullptr))
        return fail(SAT_ERR_ARG, "the plan does not fit the shared-memory resident kernel");
    p->dp.step_kernel = kind;
    return SAT_OK;
}

sat_status sat_plan_step_kernel(const sat_plan* p, int32_t act_dtype, int32_t* kind) {
    if (!p || !kind) return fail(SAT_ERR_ARG, "NULL argument");
    if (act_dtype < SAT_ACT_F32 || act_dtype > SAT_ACT_F16) return fail(SAT_ERR_ARG, "bad act_dtype");
    const bool fits = sat::resident_config(p->dp, act_dtype, nullptr, nullptr);
    if (p->dp.step_kernel == SAT_STEP_KERNEL_TILED || (p->dp.step_kernel == SAT_STEP_KERNEL_AUTO && !fits))
        *kind = SAT_STEP_KERNEL_TILED;
    else if (fits)
        *kind = SAT_STEP_KERNEL_RESIDENT;
    else
        return fail(SAT_ERR_ARG, "resident step kernel requested, but the plan does not fit it with this act_dtype");
    return SAT_OK;
}

void sat_plan_free(sat_plan* p) {
    if (!p) return;
    for (void* a : p->allocs) obj_free(a);
    for (void* a : p->lay_allocs) obj_free(a);
    delete p;
}

sat_status sat_plan_create(const sat_circuit* c, const sat_cnf* cnf, sat_plan** out) {
    if (!c || !cnf || !out) return fail(SAT_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (cnf->cnf.n_vars != c->circ.n_vars || cnf->cnf.n_clauses() != c->cnf_clauses)
        return fail(SAT_ERR_ARG, "circuit was built from a different CNF");
    const sat::Plan& P = c->plan;
    if (P.n_cone >= (1ull << 28) || P.n_nodes >= (1ull << 28))
        return fail(SAT_ERR_ARG, "circuit too large: node ids must fit in 28 bits");
    auto* p = new sat_plan();
    CK(cudaGetDevice(&p->device));
    sat_status st;
    auto bail = [&](sat_status s) { sat_plan_free(p); return s; };
    sat::DevPlan& d = p->dp;
    d.n_cone_pi = (int32_t)P.n_cone_pi;
    d.n_cone = (int64_t)P.n_cone;
    d.n_clev = (int32_t)P.c_level_off.size() - 2;
    d.max_span = (int32_t)std::max<uint32_t>(P.max_span, 1);
    d.n_out = (int32_t)P.c_out_node.size();
    d.n_pi = (int32_t)P.n_pi;
    d.n_nodes = (int64_t)P.n_nodes;
    d.n_flev = (int32_t)P.level_off.size() - 2;
    d.n_clauses = (int64_t)(P.cl_off.size() - 1);
    d.key_words = (int32_t)((P.n_pi + 31) / 32);
    std::vector<int2> cg(P.c_in0.size()), fg(P.in0.size());
    for (size_t g = 0; g < cg.size(); g++) cg[g] = make_int2(P.c_in0[g] | ((int32_t)P.c_gop[g] << 28), P.c_in1[g]);
    for (size_t g = 0; g < fg.size(); g++) fg[g] = make_int2(P.in0[g] | ((int32_t)P.gop[g] << 28), P.in1[g]);
    // Adjoint ring: a gate level's adjoints are read by the inputs of its gates, at most
    // max_span levels down, so max_span + 1 slots of the largest level hold every live one.
    {
        int32_t M = 0;
        for (int32_t l = 1; l <= d.n_clev; l++) M = std::max(M, P.c_level_off[l + 1] - P.c_level_off[l]);
        const int64_t ring = (int64_t)P.n_cone_pi + (int64_t)(d.max_span + 1) * M;
        if (d.max_span + 1 < d.n_clev && ring < (int64_t)P.n_cone) {
            d.adj_slots = d.max_span + 1;
            d.adj_slot_rows = M;
            d.n_adj_rows = ring;
        } else {
            d.n_adj_rows = (int64_t)P.n_cone;
        }
        d.seed_row = (int32_t)d.n_adj_rows;  // one more row: the seeds' scale, written per backward pass
        d.n_adj_rows += 1;
    }
    std::vector<int4> fe(P.fo_g.size());
    {
        // edge record: consumer's adj row (the seed row for an output seed or a zero edge), sibling,
        // and the partial's coefficients c0, c1 as float bits
        std::vector<int32_t> adj_row(P.n_cone);
        for (uint32_t i = 0; i < P.n_cone_pi; i++) adj_row[i] = (int32_t)i;
        for (int32_t l = 1; l <= d.n_clev; l++)
            for (int32_t x = P.c_level_off[l]; x < P.c_level_off[l + 1]; x++)
                adj_row[x] = (int32_t)(sat::adj_level_row(d, l, P.c_level_off[l]) + (x - P.c_level_off[l]));
        for (size_t e = 0; e < fe.size(); e++) {
            float c0 = (float)P.fo_c0[e], c1 = (float)P.fo_c1[e];
            int32_t i0, i1;
            std::memcpy(&i0, &c0, 4);
            std::memcpy(&i1, &c1, 4);
            fe[e] = make_int4(P.fo_g[e] < 0 ? d.seed_row : adj_row[P.fo_g[e]], P.fo_sib[e], i0, i1);
        }
    }
    // Dead adjoint rows per backward level (ring only): a gate's adjoint row is read by the
    // fan-out edges of its inputs, the last time at the level of its lowest input; it is
    // dropped from L2 after that level unless the very next level reuses its slot (its level
    // is then exactly max_span above, and the slot's new rows are written right after the
    // barrier).
    std::vector<int32_t> dead_off(d.n_clev + 2, 0), dead_row;
    if (d.adj_slots > 0) {
        auto level_of = [&](int64_t x) {
            if (x < (int64_t)P.n_cone_pi) return 0;
            return (int32_t)(std::upper_bound(P.c_level_off.begin() + 1, P.c_level_off.end(), (int32_t)x) -
                             P.c_level_off.begin()) - 1;
        };
        std::vector<int32_t> last(P.n_cone, -1);  // lowest level among each consumer's inputs
        for (size_t n = 0; n + 1 < P.fo_off.size(); n++) {
            const int32_t ln = level_of((int64_t)n);
            for (uint64_t e = P.fo_off[n]; e < P.fo_off[n + 1]; e++) {
                const int64_t g = P.fo_g[e];
                if (g >= 0 && (last[g] < 0 || ln < last[g])) last[g] = ln;
            }
        }
        std::vector<std::vector<int32_t>> per(d.n_clev + 1);
        for (int32_t L = 1; L <= d.n_clev; L++)
            for (int32_t x = P.c_level_off[L]; x < P.c_level_off[L + 1]; x++) {
                const int32_t l = last[x];
                if (l >= 0 && l < L && L - l <= d.max_span - 1)
                    per[l].push_back((int32_t)(sat::adj_level_row(d, L, P.c_level_off[L]) + (x - P.c_level_off[L])));
            }
        for (int32_t l = 0; l <= d.n_clev; l++) {
            dead_off[l] = (int32_t)dead_row.size();
            dead_row.insert(dead_row.end(), per[l].begin(), per[l].end());
        }
        dead_off[d.n_clev + 1] = (int32_t)dead_row.size();
        for (int32_t r : dead_row)
            if (r < (int32_t)P.n_cone_pi || r >= d.seed_row)
                return bail(fail(SAT_ERR_ARG, "internal error: dead adjoint row outside the ring"));
    }
    // Adjoint node runs balanced by fan-out edges, one table per warp count of the step
    // kernels: warp w of W starts at the first node of the level whose edges begin at or
    // after w / W of the level's edges.
    std::vector<int32_t> adj_run;
    {
        int32_t counts[sat::DevPlan::ADJ_RUN_SETS];
        sat::step_warp_counts(counts);
        for (int k = 0; k < sat::DevPlan::ADJ_RUN_SETS; k++) {
            const int32_t W = counts[k];
            d.adj_run_w[k] = W;
            d.adj_run_base[k] = (int64_t)adj_run.size();
            for (int32_t l = 0; l <= d.n_clev; l++) {
                const int64_t lo = l == 0 ? 0 : P.c_level_off[l];
                const int64_t hi = l == 0 ? (int64_t)P.n_cone_pi : P.c_level_off[l + 1];
                const int64_t e0 = (int64_t)P.fo_off[lo], E = (int64_t)P.fo_off[hi] - e0;
                int64_t prev = lo;
                for (int32_t w = 0; w <= W; w++) {
                    int64_t u = hi;
                    if (w < W) {
                        const int64_t target = e0 + E * w / W;
                        u = std::lower_bound(P.fo_off.begin() + lo, P.fo_off.begin() + hi, target) - P.fo_off.begin();
                    }
                    u = std::max(u, prev);
                    adj_run.push_back((int32_t)u);
                    prev = u;
                }
            }
        }
    }
    // bit 31 of the sibling field marks the last edge of each node's range
    for (size_t n = 0; n + 1 < P.fo_off.size(); n++)
        if (P.fo_off[n + 1] > P.fo_off[n]) fe[(size_t)P.fo_off[n + 1] - 1].y |= (int32_t)0x80000000u;
    if (!records_in_range(cg, fe, P.c_out_node, (int64_t)P.n_cone, d.n_adj_rows))
        return bail(fail(SAT_ERR_ARG, "internal error: plan records outside the scratch block"));
    std::vector<int32_t> cl_lit(P.cl_node.size());
    for (size_t i = 0; i < cl_lit.size(); i++) cl_lit[i] = (P.cl_node[i] << 1) | P.cl_neg[i];
    if ((st = upload(p, P.c_level_off, &d.c_level_off)) != SAT_OK) return bail(st);
    if ((st = upload(p, cg, &d.c_gate)) != SAT_OK) return bail(st);
    if ((st = upload(p, P.cone_pi_row, &d.cone_pi_row)) != SAT_OK) return bail(st);
    if (P.fo_g.size() >= (1ull << 31)) return bail(fail(SAT_ERR_ARG, "too many fan-out edges (limit 2^31)"));
    std::vector<int32_t> fo_off32(P.fo_off.begin(), P.fo_off.end());
    if ((st = upload(p, fo_off32, &d.fo_off)) != SAT_OK) return bail(st);
    if ((st = upload(p, fe, &d.fo_edge)) != SAT_OK) return bail(st);
    if ((st = upload(p, P.c_out_node, &d.c_out_node)) != SAT_OK) return bail(st);
    if ((st = upload(p, P.out_target, &d.out_target)) != SAT_OK) return bail(st);
    if ((st = upload(p, P.level_off, &d.f_level_off)) != SAT_OK) return bail(st);
    if ((st = upload(p, fg, &d.f_gate)) != SAT_OK) return bail(st);
    if ((st = upload(p, P.cl_off, &d.cl_off)) != SAT_OK) return bail(st);
    if ((st = upload(p, cl_lit, &d.cl_lit)) != SAT_OK) return bail(st);
    if ((st = upload(p, adj_run, &d.adj_run)) != SAT_OK) return bail(st);
    if (!dead_row.empty()) {
        if ((st = upload(p, dead_off, &d.dead_off)) != SAT_OK) return bail(st);
        if ((st = upload(p, dead_row, &d.dead_row)) != SAT_OK) return bail(st);
    }
    d.full.k = 0;
    d.full.n_act_rows = (int64_t)P.n_cone;
    d.full.act_off = d.c_level_off;
    d.full.gate = d.c_gate;
    d.full.edge = d.fo_edge;
    d.full.out_row = d.c_out_node;
    p->h_gate = std::move(cg);
    p->h_edge = std::move(fe);
    p->h_out = P.c_out_node;
    {
        void* w = nullptr;
        if (!obj_alloc(&w, sizeof(unsigned int)))
            return bail(fail(SAT_ERR_OOM, "device allocation failed for the status word"));
        p->allocs.push_back(w);
        d.status = (unsigned int*)w;
        CK(cudaMemset(w, 0, sizeof(unsigned int)));
    }
    p->h_c_level_off = P.c_level_off;
    p->h_f_level_off = P.level_off;
    d.h_c_level_off = p->h_c_level_off.data();
    d.h_f_level_off = p->h_f_level_off.data();
    p->pi_var = P.pi_var;
    p->var_cone.assign(P.n_vars + 1, -1);
    p->var_full.assign(P.n_vars + 1, -1);
    p->var_neg.assign(P.n_vars + 1, 0);
    {
        // full node -> cone index
        std::vector<int64_t> f2c(P.n_nodes, -1);
        for (uint32_t i = 0; i < P.n_cone_pi; i++) f2c[P.cone_pi_row[i]] = i;
        uint64_t ci = P.n_cone_pi;
        std::vector<uint8_t> cone(P.n_nodes, 0);
        // cone gates are the full gates in order that belong to the cone: rebuild by walking outputs
        for (int32_t n : P.out_node) cone[n] = 1;
        for (int64_t r = (int64_t)P.in0.size() - 1; r >= 0; r--)
            if (cone[P.n_pi + r]) cone[P.in0[r]] = cone[P.in1[r]] = 1;
        for (size_t r = 0; r < P.in0.size(); r++)
            if (cone[P.n_pi + r]) f2c[P.n_pi + r] = (int64_t)ci++;
        for (uint32_t v = 1; v <= P.n_vars; v++) {
            p->var_full[v] = P.var_node[v];
            p->var_cone[v] = f2c[P.var_node[v]];
            p->var_neg[v] = P.var_neg[v];
        }
    }
    p->f_in0 = P.in0;
    p->f_in1 = P.in1;
    p->f_gop = P.gop;
    sat_plan_info& I = p->info;  // upload_bytes was accumulated by upload()
    I.n_vars = P.n_vars;
    I.n_pi = P.n_pi;
    I.n_cone_pi = P.n_cone_pi;
    I.n_outputs = (uint32_t)P.out_node.size();
    I.n_cone_levels = (uint32_t)d.n_clev;
    I.n_levels = (uint32_t)d.n_flev;
    I.key_words = (uint32_t)d.key_words;
    I.max_span = P.max_span;
    I.n_cone = P.n_cone;
    I.n_nodes = P.n_nodes;
    I.n_cone_gates = P.c_in0.size();
    I.n_gates = P.in0.size();
    I.n_clauses = (uint64_t)d.n_clauses;
    I.n_fanout_edges = P.fo_g.size();
    if (sat::round_kernel_fits(P, nullptr)) {
        p->round.reset(new sat::CompiledRound());
        p->round->source = sat::round_kernel_source(P);
    }
    *out = p;
    return SAT_OK;
}

sat_status sat_plan_round_info(const sat_plan* p, int32_t compile, sat_round_info* info) {
    if (!p || !info) return fail(SAT_ERR_ARG, "NULL argument");
    *info = sat_round_info{};
    if (!p->round) return SAT_OK;
    info->available = 1;
    if (compile) {
        sat_status s = check_device(p->device);
        if (s != SAT_OK) return s;
        std::string err;
        if (p->round->ensure(err) != cudaSuccess) return fail(SAT_ERR_CUDA, err);
    }
    std::lock_guard<std::mutex> g(p->round->mu);
    if (p->round->mod) {
        info->compiled = 1;
        info->registers = p->round->mod->registers;
        info->spill_bytes = p->round->mod->spill_bytes;
        info->min_blocks = p->round->mod->min_blocks;
        info->compile_ms = p->round->mod->compile_ms;
    }
    return SAT_OK;
}

sat_status sat_round_gd(const sat_plan* p, float lr, int32_t n_steps, uint64_t seed, uint32_t round,
                        float init_scale, float* V, int64_t ldv, uint32_t* keys, uint32_t* valid, int64_t B,
                        void* stream) {
    sat_status s = sat::check_plan_call(p, B, V ? ldv : -1);
    if (s != SAT_OK) return s;
    if (!keys || !valid) return fail(SAT_ERR_ARG, "NULL keys or valid");
    if (n_steps < 0 || !std::isfinite(lr) || !std::isfinite(init_scale))
        return fail(SAT_ERR_ARG, "n_steps must be >= 0, lr and init_scale finite");
    if (!p->round) return fail(SAT_ERR_ARG, "the plan's circuit exceeds the compiled round kernel's limits");
    std::string err;
    if (p->round->ensure(err) != cudaSuccess) return fail(SAT_ERR_CUDA, err);
    // the round kernel writes the cone inputs' final logits; every other input keeps its
    // initial one, which the init kernel writes first
    if (V) CK(sat::launch_init_normal(p->dp, seed, round, init_scale, V, ldv, B, S(stream)));
    CK(p->round->launch(seed, round, init_scale, lr, n_steps, V, ldv, keys, valid, B, S(stream)));
    return SAT_OK;
}

sat_status sat_plan_status(const sat_plan* p, uint32_t* status, int32_t clear, void* stream) {
    if (!p || !status) return fail(SAT_ERR_ARG, "NULL argument");
    unsigned int v = 0;
    CK(cudaMemcpyAsync(&v, p->dp.status, sizeof(v), cudaMemcpyDeviceToHost, S(stream)));
    if (clear) CK(cudaMemsetAsync(p->dp.status, 0, sizeof(v), S(stream)));
    CK(cudaStreamSynchronize(S(stream)));
    *status = v;
    return SAT_OK;
}

sat_status sat_plan_get_info(const sat_plan* p, sat_plan_info* info) {
    if (!p || !info) return fail(SAT_ERR_ARG, "NULL argument");
    *info = p->info;
    return SAT_OK;
}

sat_status sat_plan_scratch_elems(const sat_plan* p, int64_t B, uint64_t* elems) {
    if (!p || !elems || B < 0) return fail(SAT_ERR_ARG, "bad argument");
    const uint64_t rows = std::max<uint64_t>(p->info.n_cone, (uint64_t)p->dp.n_adj_rows);
    *elems = (uint64_t)((B + SAT_TILE_SAMPLES - 1) / SAT_TILE_SAMPLES) * rows * SAT_TILE_SAMPLES;
    return SAT_OK;
}

// The act layout of segment length k (0: the full layout), built and uploaded on first use.
// Levels 1.. form segments of k levels (segment j = levels jk+1 .. jk+k).  Kept levels:
// 0, the top max_span levels of each segment (every input of the next segment's gates is
// among them, since no edge spans more than max_span levels) and levels with an output
// (the loss reads them).  Kept levels get their own rows; the other levels of segment j
// go to scratch buffer j % 2, which holds the largest segment's unkept levels.
static sat_status plan_layout(const sat_plan* p, int32_t k, const sat::DevAct** out) {
    *out = nullptr;
    if (k < 0) return fail(SAT_ERR_ARG, "segment must be >= 0");
    if (k == 0) {
        *out = &p->dp.full;
        return SAT_OK;
    }
    std::lock_guard<std::mutex> lock(p->lay_mu);
    auto it = p->layouts.find(k);
    if (it != p->layouts.end()) {
        *out = &it->second;
        return SAT_OK;
    }
    const sat::DevPlan& d = p->dp;
    const std::vector<int32_t>& off = p->h_c_level_off;
    const int32_t L = d.n_clev, W = d.max_span;
    std::vector<int32_t> level(d.n_cone, 0);
    for (int32_t l = 1; l <= L; l++)
        for (int32_t x = off[l]; x < off[l + 1]; x++) level[x] = l;
    std::vector<uint8_t> stored(L + 1, 0);
    stored[0] = 1;
    for (int32_t l = 1; l <= L; l++) stored[l] = (uint8_t)((l - 1) % k >= k - W);
    for (int32_t x : p->h_out) stored[level[x]] = 1;
    std::vector<int32_t> act_off(L + 1, 0);
    int64_t next = d.n_cone_pi;
    for (int32_t l = 1; l <= L; l++)
        if (stored[l]) {
            act_off[l] = (int32_t)next;
            next += off[l + 1] - off[l];
        }
    int64_t S = 0;
    for (int64_t l0 = 1; l0 <= L; l0 += k) {
        int64_t seg = 0;
        for (int64_t l = l0; l < l0 + k && l <= L; l++)
            if (!stored[l]) seg += off[l + 1] - off[l];
        S = std::max(S, seg);
    }
    for (int64_t l0 = 1, j = 0; l0 <= L; l0 += k, j++) {
        int64_t pos = next + (j % 2) * S;
        for (int64_t l = l0; l < l0 + k && l <= L; l++)
            if (!stored[l]) {
                act_off[l] = (int32_t)pos;
                pos += off[l + 1] - off[l];
            }
    }
    auto row = [&](int32_t x) { return x < d.n_cone_pi ? x : act_off[level[x]] + (x - off[level[x]]); };
    std::vector<int2> gate(p->h_gate.size());
    for (size_t g = 0; g < gate.size(); g++) {
        const int2 r = p->h_gate[g];
        gate[g] = make_int2(row(r.x & 0x0FFFFFFF) | (int32_t)((uint32_t)r.x & 0xF0000000u), row(r.y));
    }
    std::vector<int4> edge(p->h_edge);
    for (int4& e : edge) e.y = row(e.y & 0x7FFFFFFF) | (int32_t)((uint32_t)e.y & 0x80000000u);
    std::vector<int32_t> out_row(p->h_out.size());
    for (size_t j = 0; j < out_row.size(); j++) out_row[j] = row(p->h_out[j]);
    if (next + 2 * S >= d.n_cone) {  // no saving (segments too long or too short): keep every level
        *out = &(p->layouts[k] = d.full);
        return SAT_OK;
    }
    sat::DevAct a;
    a.k = k;
    a.n_act_rows = next + 2 * S;
    if (!records_in_range(gate, edge, out_row, a.n_act_rows, d.n_adj_rows))
        return fail(SAT_ERR_ARG, "internal error: recomputation records outside the scratch block");
    sat_status st;
    if ((st = upload_to(p->lay_allocs, act_off, &a.act_off)) != SAT_OK) return st;
    if ((st = upload_to(p->lay_allocs, stored, &a.stored)) != SAT_OK) return st;
    if ((st = upload_to(p->lay_allocs, gate, &a.gate)) != SAT_OK) return st;
    if ((st = upload_to(p->lay_allocs, edge, &a.edge)) != SAT_OK) return st;
    if ((st = upload_to(p->lay_allocs, out_row, &a.out_row)) != SAT_OK) return st;
    *out = &(p->layouts[k] = a);
    return SAT_OK;
}

sat_status sat_plan_layout_elems(const sat_plan* p, int32_t segment, int64_t B, uint64_t* act_elems,
                                 uint64_t* adj_elems) {
    if (!p || B < 0) return fail(SAT_ERR_ARG, "bad argument");
    if (segment < 0) return fail(SAT_ERR_ARG, "segment must be >= 0");
    const uint64_t tiles = (uint64_t)((B + SAT_TILE_SAMPLES - 1) / SAT_TILE_SAMPLES);
    if (act_elems) {
        sat_status st = segment > 0 ? check_device(p->device) : SAT_OK;
        if (st != SAT_OK) return st;
        const sat::DevAct* lay = nullptr;
        if ((st = plan_layout(p, segment, &lay)) != SAT_OK) return st;
        *act_elems = tiles * (uint64_t)lay->n_act_rows * SAT_TILE_SAMPLES;
    }
    if (adj_elems) *adj_elems = tiles * (uint64_t)p->dp.n_adj_rows * SAT_TILE_SAMPLES;
    return SAT_OK;
}

sat_status sat_diag_bounded_wait(uint32_t limit_us, uint32_t* status, void* stream) {
    if (!status || limit_us == 0 || limit_us > 10000000u)
        return fail(SAT_ERR_ARG, "bad argument (limit_us in 1..10^7, status non-NULL)");
    unsigned* d = nullptr;
    if (cudaMalloc(&d, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return fail(SAT_ERR_OOM, "cudaMalloc failed for the status word");
    }
    unsigned h = 0;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned), S(stream));
    if (e == cudaSuccess) e = sat::launch_bounded_wait_diag(d, (uint64_t)limit_us * 1000u, S(stream));
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(unsigned), cudaMemcpyDeviceToHost, S(stream));
    if (e == cudaSuccess) e = cudaStreamSynchronize(S(stream));
    cudaFree(d);
    if (e != cudaSuccess) return fail(SAT_ERR_CUDA, std::string("diagnostic kernel: ") + cudaGetErrorString(e));
    *status = h;
    return SAT_OK;
}

sat_status sat_diag_angle_signs(uint32_t* mismatches, void* stream) {
    if (!mismatches) return fail(SAT_ERR_ARG, "NULL argument");
    unsigned* d = nullptr;
    if (cudaMalloc(&d, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return fail(SAT_ERR_OOM, "cudaMalloc failed for the counter");
    }
    unsigned h = 0;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned), S(stream));
    if (e == cudaSuccess) e = sat::launch_angle_signs_diag(d, S(stream));
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(unsigned), cudaMemcpyDeviceToHost, S(stream));
    if (e == cudaSuccess) e = cudaStreamSynchronize(S(stream));
    cudaFree(d);
    if (e != cudaSuccess) return fail(SAT_ERR_CUDA, std::string("diagnostic kernel: ") + cudaGetErrorString(e));
    *mismatches = h;
    return SAT_OK;
}

sat_status sat_plan_pi_vars(const sat_plan* p, uint32_t* vars) {
    if (!p || !vars) return fail(SAT_ERR_ARG, "NULL argument");
    std::copy(p->pi_var.begin(), p->pi_var.end(), vars);
    return SAT_OK;
}

sat_status sat_mlp_train(sat_mlp* m, const sat_plan* p, const uint64_t* sols, uint64_t n, int32_t steps, int64_t nb,
                         int32_t K, float lr, uint64_t seed, float* loss_host, void* stream) {
    if (!m || !p || (!sols && n > 0) || steps < 0 || nb < 1 || K < 1 || !(lr > 0.0f))
        return fail(SAT_ERR_ARG, "bad argument (S, K >= 1, lr > 0, steps >= 0)");
    if (n == 0 || steps == 0) return SAT_OK;
    const size_t n_pi = p->pi_var.size(), kw = (n_pi + 31) / 32, aw = (p->info.n_vars + 63) / 64;
    if (n_pi == 0) return fail(SAT_ERR_ARG, "the plan has no primary inputs");
    // targets: the primary-input bits of every solution, packed like the sampler's keys
    std::vector<uint32_t> keys(n * kw, 0u);
    for (uint64_t s = 0; s < n; s++)
        for (size_t i = 0; i < n_pi; i++) {
            const uint32_t v = p->pi_var[i] - 1;  // DIMACS var v -> bit v-1 of the assignment
            if ((sols[s * aw + v / 64] >> (v % 64)) & 1ull) keys[s * kw + i / 32] |= 1u << (i % 32);
        }
    cudaStream_t str = S(stream);
    uint32_t* d_batch = nullptr;
    struct Free {
        void* a;
        ~Free() { cudaFree(a); }
    } fr{nullptr};
    if (cudaMalloc(&d_batch, (size_t)nb * kw * 4) != cudaSuccess) return fail(SAT_ERR_OOM, "cudaMalloc failed (batch)");
    fr.a = d_batch;
    std::vector<uint32_t> batch((size_t)nb * kw);
    uint64_t state = seed;
    auto next = [&state]() {  // SplitMix64
        uint64_t z = (state += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    for (int32_t it = 0; it < steps; it++) {
        for (int64_t j = 0; j < nb; j++) {
            const uint64_t r = next() % n;
            std::copy(keys.begin() + r * kw, keys.begin() + (r + 1) * kw, batch.begin() + j * kw);
        }
        // pageable source: staged before the call returns, so the buffer is reused safely
        CK(cudaMemcpyAsync(d_batch, batch.data(), batch.size() * 4, cudaMemcpyHostToDevice, str));
        sat_status s = sat_mlp_train_step(m, d_batch, (int32_t)kw, nb, K, lr, seed, (uint32_t)it,
                                          it + 1 == steps ? loss_host : nullptr, stream);
        if (s != SAT_OK) return s;
    }
    CK(cudaStreamSynchronize(str));
    return SAT_OK;
}

sat_status sat_plan_var_nodes(const sat_plan* p, int64_t* cone_node, int64_t* full_node, uint8_t* neg) {
    if (!p) return fail(SAT_ERR_ARG, "NULL plan");
    if (cone_node) std::copy(p->var_cone.begin(), p->var_cone.end(), cone_node);
    if (full_node) std::copy(p->var_full.begin(), p->var_full.end(), full_node);
    if (neg) std::copy(p->var_neg.begin(), p->var_neg.end(), neg);
    return SAT_OK;
}

// -------------------------------------------------------------- kernels --
sat_status sat_init_normal(const sat_plan* p, uint64_t seed, uint32_t round, float scale, float* V, int64_t ldv,
                           int64_t B, void* stream) {
    sat_status s = check_layout(p, B, ldv);
    if (s != SAT_OK) return s;
    if (B > 0 && p->dp.n_pi > 0 && !V) return fail(SAT_ERR_ARG, "V is NULL");
    CK(sat::launch_init_normal(p->dp, seed, round, scale, V, ldv, B, S(stream)));
    return SAT_OK;
}

sat_status sat_forward(const sat_plan* p, sat_act_dtype t, const float* V, int64_t ldv, void* act, float* loss,
                       int64_t B, void* stream) {
    sat_status s = check_layout(p, B, ldv);
    if (s != SAT_OK) return s;
    if (t < SAT_ACT_F32 || t > SAT_ACT_F16) return fail(SAT_ERR_ARG, "bad act_dtype");
    if (B > 0 && ((p->dp.n_pi > 0 && !V) || (p->dp.n_cone > 0 && !act))) return fail(SAT_ERR_ARG, "NULL buffer");
    if (((uintptr_t)act & 15) != 0) return fail(SAT_ERR_ARG, "act must be 16-byte aligned");
    CK(sat::launch_forward(p->dp, (int)t, V, ldv, act, loss, B, S(stream)));
    return SAT_OK;
}

sat_status sat_backward(const sat_plan* p, sat_act_dtype t, const float* V, int64_t ldv, const void* act, float* adj,
                        const float* grad_loss, float* gV, int64_t B, void* stream) {
    sat_status s = check_layout(p, B, ldv);
    if (s != SAT_OK) return s;
    if (t < SAT_ACT_F32 || t > SAT_ACT_F16) return fail(SAT_ERR_ARG, "bad act_dtype");
    if (B > 0 && ((p->dp.n_pi > 0 && (!V || !gV)) || (p->dp.n_cone > 0 && (!act || !adj))))
        return fail(SAT_ERR_ARG, "NULL buffer");
    if ((((uintptr_t)act | (uintptr_t)adj) & 15) != 0) return fail(SAT_ERR_ARG, "act/adj must be 16-byte aligned");
    CK(sat::launch_backward(p->dp, (int)t, V, ldv, act, adj, grad_loss, gV, B, S(stream)));
    return SAT_OK;
}

sat_status sat_opt_update(const sat_plan* p, const sat_opt_params* o, float* V, float* m, float* v, const float* gV,
                          int64_t ldv, int32_t t, int64_t B, void* stream) {
    sat_status s = check_layout(p, B, ldv);
    if (s != SAT_OK) return s;
    if (!opt_ok(o) || t < 1) return fail(SAT_ERR_ARG, "bad optimiser parameters or step");
    if (B > 0 && p->dp.n_cone_pi > 0 && (!V || !gV || (o->optimizer == SAT_OPT_ADAM && (!m || !v))))
        return fail(SAT_ERR_ARG, "NULL buffer");
    CK(sat::launch_opt_update(p->dp, opt_of(o), V, m, v, gV, ldv, t, B, S(stream)));
    return SAT_OK;
}

sat_status sat_steps(const sat_plan* p, sat_act_dtype t, const sat_opt_params* o, float* V, float* m, float* v,
                     int64_t ldv, void* act, float* adj, float* loss, int32_t t0, int32_t n_steps, int64_t B,
                     void* stream) {
    sat_status s = check_layout(p, B, ldv);
    if (s != SAT_OK) return s;
    if (t < SAT_ACT_F32 || t > SAT_ACT_F16) return fail(SAT_ERR_ARG, "bad act_dtype");
    if (!opt_ok(o) || t0 < 1 || n_steps < 0) return fail(SAT_ERR_ARG, "bad optimiser parameters or steps");
    if (B > 0 && ((p->dp.n_pi > 0 && (!V || (o->optimizer == SAT_OPT_ADAM && (!m || !v)))) ||
                  (p->dp.n_cone > 0 && (!act || !adj))))
        return fail(SAT_ERR_ARG, "NULL buffer");
    if ((((uintptr_t)act | (uintptr_t)adj) & 15) != 0) return fail(SAT_ERR_ARG, "act/adj must be 16-byte aligned");
    CK(sat::launch_steps(p->dp, p->dp.full, (int)t, opt_of(o), V, m, v, ldv, act, adj, loss, t0, n_steps, B,
                         S(stream)));
    return SAT_OK;
}

sat_status sat_steps_aged(const sat_plan* p, sat_act_dtype t, const sat_opt_params* o, float* V, float* m, float* v,
                          int64_t ldv, void* act, float* adj, float* loss, const int32_t* age, int32_t t0,
                          int32_t n_steps, int64_t B, void* stream) {
    sat_status s = check_layout(p, B, ldv);
    if (s != SAT_OK) return s;
    if (t < SAT_ACT_F32 || t > SAT_ACT_F16) return fail(SAT_ERR_ARG, "bad act_dtype");
    if (!opt_ok(o) || t0 < 1 || n_steps < 0) return fail(SAT_ERR_ARG, "bad optimiser parameters or steps");
    if (B > 0 && ((p->dp.n_pi > 0 && (!V || (o->optimizer == SAT_OPT_ADAM && (!m || !v)))) ||
                  (p->dp.n_cone > 0 && (!act || !adj))))
        return fail(SAT_ERR_ARG, "NULL buffer");
    if ((((uintptr_t)act | (uintptr_t)adj) & 15) != 0) return fail(SAT_ERR_ARG, "act/adj must be 16-byte aligned");
    CK(sat::launch_steps(p->dp, p->dp.full, (int)t, opt_of(o), V, m, v, ldv, act, adj, loss, t0, n_steps, B,
                         S(stream), age));
    return SAT_OK;
}

sat_status sat_steps_recompute(const sat_plan* p, sat_act_dtype t, const sat_opt_params* o, float* V, float* m,
                               float* v, int64_t ldv, void* act, float* adj, float* loss, const int32_t* age,
                               int32_t t0, int32_t n_steps, int64_t B, int32_t segment, void* stream) {
    sat_status s = check_layout(p, B, ldv);
    if (s != SAT_OK) return s;
    if (t < SAT_ACT_F32 || t > SAT_ACT_F16) return fail(SAT_ERR_ARG, "bad act_dtype");
    if (!opt_ok(o) || t0 < 1 || n_steps < 0) return fail(SAT_ERR_ARG, "bad optimiser parameters or steps");
    if (segment < 0) return fail(SAT_ERR_ARG, "segment must be >= 0");
    if (B > 0 && ((p->dp.n_pi > 0 && (!V || (o->optimizer == SAT_OPT_ADAM && (!m || !v)))) ||
                  (p->dp.n_cone > 0 && (!act || !adj))))
        return fail(SAT_ERR_ARG, "NULL buffer");
    if ((((uintptr_t)act | (uintptr_t)adj) & 15) != 0) return fail(SAT_ERR_ARG, "act/adj must be 16-byte aligned");
    const sat::DevAct* lay = nullptr;
    if ((s = plan_layout(p, segment, &lay)) != SAT_OK) return s;
    CK(sat::launch_steps(p->dp, *lay, (int)t, opt_of(o), V, m, v, ldv, act, adj, loss, t0, n_steps, B, S(stream),
                         age));
    return SAT_OK;
}

sat_status sat_retire(const uint32_t* valid, int32_t* age, uint32_t* restart, int32_t k, int32_t max_age, int64_t B,
                      void* stream) {
    if (B < 0 || k < 0 || max_age < 1) return fail(SAT_ERR_ARG, "bad k / max_age / batch");
    if (B > 0 && (!valid || !age || !restart)) return fail(SAT_ERR_ARG, "NULL buffer");
    CK(sat::launch_retire(valid, age, restart, k, max_age, B, S(stream)));
    return SAT_OK;
}

sat_status sat_restart(const sat_plan* p, const uint32_t* restart, uint64_t seed, uint32_t round, float init_scale,
                       const float* src, int64_t lds, float* V, float* m, float* v, int64_t ldv, int64_t B,
                       void* stream) {
    sat_status s = check_layout(p, B, ldv);
    if (s != SAT_OK) return s;
    if (src && lds < B) return fail(SAT_ERR_ARG, "lds < batch");
    if (B > 0 && p->dp.n_pi > 0 && (!restart || !V || !m || !v)) return fail(SAT_ERR_ARG, "NULL buffer");
    CK(sat::launch_restart(p->dp, restart, seed, round, init_scale, src, lds, V, m, v, ldv, B, S(stream)));
    return SAT_OK;
}

sat_status sat_threshold(const sat_plan* p, const float* V, int64_t ldv, uint32_t* node_bits, int64_t ldw,
                         uint32_t* keys, int64_t B, void* stream) {
    sat_status s = check_layout(p, B, ldv);
    if (s != SAT_OK) return s;
    if (ldw < (B + 31) / 32) return fail(SAT_ERR_ARG, "ldw < ceil(B/32)");
    if (B > 0 && p->dp.n_pi > 0 && (!V || !node_bits || !keys)) return fail(SAT_ERR_ARG, "NULL buffer");
    CK(sat::launch_threshold(p->dp, V, ldv, node_bits, ldw, keys, B, S(stream)));
    return SAT_OK;
}

sat_status sat_hard_eval(const sat_plan* p, uint32_t* node_bits, int64_t ldw, int64_t B, void* stream) {
    sat_status s = check_layout(p, B, -1);
    if (s != SAT_OK) return s;
    if (ldw < (B + 31) / 32) return fail(SAT_ERR_ARG, "ldw < ceil(B/32)");
    if (B > 0 && p->dp.n_nodes > 0 && !node_bits) return fail(SAT_ERR_ARG, "NULL buffer");
    CK(sat::launch_hard_eval(p->dp, node_bits, ldw, B, S(stream)));
    return SAT_OK;
}

sat_status sat_cnf_check(const sat_plan* p, const uint32_t* node_bits, int64_t ldw, uint32_t* valid, int64_t B,
                         void* stream) {
    sat_status s = check_layout(p, B, -1);
    if (s != SAT_OK) return s;
    if (ldw < (B + 31) / 32) return fail(SAT_ERR_ARG, "ldw < ceil(B/32)");
    if (B > 0 && (!valid || (p->dp.n_nodes > 0 && !node_bits))) return fail(SAT_ERR_ARG, "NULL buffer");
    CK(sat::launch_cnf_check(p->dp, node_bits, ldw, valid, B, S(stream)));
    return SAT_OK;
}

// --------------------------------------------------------------- dedup --
void sat_dedup_free(sat_dedup* d) {
    if (!d) return;
    obj_free(d->d.slots);
    obj_free(d->d.pool);
    obj_free(d->d.count);
    obj_free(d->d.status);
    obj_free(d->slot_of);
    delete d;
}

sat_status sat_dedup_create(const sat_plan* p, uint64_t max_keys, int64_t max_batch, sat_dedup** out) {
    if (!p || !out || max_batch < 0) return fail(SAT_ERR_ARG, "bad argument");
    *out = nullptr;
    if (max_keys >= (1ull << 31)) return fail(SAT_ERR_ARG, "max_keys must be < 2^31");
    auto* d = new sat_dedup();
    d->device = p->device;
    d->max_batch = max_batch;
    d->d.key_words = p->dp.key_words;
    uint64_t cap = 1024;
    while (cap < 2 * std::max<uint64_t>(max_keys, 1)) cap <<= 1;
    d->d.capacity = cap;
    d->d.pool_capacity = max_keys;
    d->d.max_probe = (uint32_t)std::min<uint64_t>(cap, 1u << 20);
    const size_t kw = (size_t)std::max(1, d->d.key_words);
    if (!obj_alloc((void**)&d->d.slots, cap * sizeof(unsigned long long)) ||
        !obj_alloc((void**)&d->d.pool, std::max<uint64_t>(max_keys, 1) * kw * sizeof(uint32_t)) ||
        !obj_alloc((void**)&d->d.count, sizeof(unsigned long long)) ||
        !obj_alloc((void**)&d->d.status, sizeof(unsigned int)) ||
        !obj_alloc((void**)&d->slot_of, std::max<int64_t>(max_batch, 1) * sizeof(unsigned long long))) {
        sat_dedup_free(d);
        return fail(SAT_ERR_OOM, "device allocation failed for the dedup table");
    }
    cudaError_t e = sat::launch_dedup_clear(d->d, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) {
        sat_dedup_free(d);
        return fail(SAT_ERR_CUDA, cudaGetErrorString(e));
    }
    *out = d;
    return SAT_OK;
}

sat_status sat_dedup_clear(sat_dedup* d, void* stream) {
    if (!d) return fail(SAT_ERR_ARG, "NULL dedup");
    CK(sat::launch_dedup_clear(d->d, S(stream)));
    return SAT_OK;
}

sat_status sat_dedup_count(const sat_dedup* d, uint64_t* n, void* stream) {
    if (!d || !n) return fail(SAT_ERR_ARG, "NULL argument");
    unsigned long long c = 0;
    CK(cudaMemcpyAsync(&c, d->d.count, sizeof(c), cudaMemcpyDeviceToHost, S(stream)));
    CK(cudaStreamSynchronize(S(stream)));
    *n = std::min<uint64_t>(c, d->d.pool_capacity);
    return SAT_OK;
}

sat_status sat_dedup_insert(sat_dedup* d, const uint32_t* keys, const uint32_t* valid, int64_t B, uint64_t* hashes,
                            uint8_t* is_new, void* stream) {
    if (!d) return fail(SAT_ERR_ARG, "NULL dedup");
    if (B < 0 || B > d->max_batch) return fail(SAT_ERR_ARG, "B outside 0..max_batch");
    if (B > 0 && (!keys || !valid)) return fail(SAT_ERR_ARG, "NULL buffer");
    sat_status s = check_device(d->device);
    if (s != SAT_OK) return s;
    uint64_t n = 0;
    if ((s = sat_dedup_count(d, &n, stream)) != SAT_OK) return s;
    if (n + (uint64_t)B > d->d.pool_capacity)
        return fail(SAT_ERR_TABLE_FULL, "dedup table cannot take another batch of this size");
    CK(sat::launch_dedup_insert(d->d, keys, valid, B, (unsigned long long*)hashes, is_new, d->slot_of, S(stream)));
    unsigned int status = 0;
    CK(cudaMemcpyAsync(&status, d->d.status, sizeof(status), cudaMemcpyDeviceToHost, S(stream)));
    CK(cudaStreamSynchronize(S(stream)));
    if (status) return fail(SAT_ERR_TABLE_FULL, "dedup probe limit reached");
    return SAT_OK;
}

sat_status sat_dedup_insert_async(sat_dedup* d, const uint32_t* keys, const uint32_t* valid, int64_t B,
                                  void* stream) {
    if (!d) return fail(SAT_ERR_ARG, "NULL dedup");
    if (B < 0 || B > d->max_batch) return fail(SAT_ERR_ARG, "B outside 0..max_batch");
    if (B > 0 && (!keys || !valid)) return fail(SAT_ERR_ARG, "NULL buffer");
    sat_status s = check_device(d->device);
    if (s != SAT_OK) return s;
    // the commit kernel refuses slots past the pool's capacity (status bit 1) and the insert
    // kernel stops at the probe limit (bit 0): nothing is written out of bounds
    CK(sat::launch_dedup_insert(d->d, keys, valid, B, nullptr, nullptr, d->slot_of, S(stream)));
    return SAT_OK;
}

sat_status sat_dedup_check(const sat_dedup* d, void* stream) {
    if (!d) return fail(SAT_ERR_ARG, "NULL dedup");
    unsigned int status = 0;
    CK(cudaMemcpyAsync(&status, d->d.status, sizeof(status), cudaMemcpyDeviceToHost, S(stream)));
    CK(cudaStreamSynchronize(S(stream)));
    if (status) return fail(SAT_ERR_TABLE_FULL, "dedup table full or probe limit reached");
    return SAT_OK;
}

sat_status sat_dedup_copy_keys(const sat_dedup* d, uint64_t first, uint64_t count, uint32_t* host_keys,
                               void* stream) {
    if (!d || (count && !host_keys)) return fail(SAT_ERR_ARG, "NULL argument");
    uint64_t n = 0;
    sat_status s = sat_dedup_count(d, &n, stream);
    if (s != SAT_OK) return s;
    if (first + count > n) return fail(SAT_ERR_ARG, "range beyond stored keys");
    const size_t kw = (size_t)d->d.key_words;
    if (count && kw) {
        CK(cudaMemcpyAsync(host_keys, d->d.pool + first * kw, count * kw * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                           S(stream)));
        CK(cudaStreamSynchronize(S(stream)));
    }
    return SAT_OK;
}

// ----------------------------------------------------------- end to end --
void sat_sample_opts_default(sat_sample_opts* o) {
    if (!o) return;
    *o = sat_sample_opts{};
    o->batch = 1024;
    o->steps = 200;
    o->max_rounds = 1;
    o->opt.optimizer = SAT_OPT_ADAM;
    o->opt.lr = 0.1f;
    o->opt.beta1 = 0.9f;
    o->opt.beta2 = 0.999f;
    o->opt.eps = 1e-8f;
    o->seed = 0;
    o->first_round = 0;
    o->init_scale = 1.0f;
    o->act_dtype = SAT_ACT_F32;
    o->steps_per_launch = 0;
    o->init_logits = nullptr;
    o->init_ld = 0;
    o->stream = nullptr;
    o->proposal = nullptr;
    o->proposal_tau = 1.0f;
    o->check_every = 0;
    o->max_age = 0;
    o->recompute_segment = 0;
    o->step_kernel = SAT_STEP_KERNEL_AUTO;
}

namespace {


// A pinned host buffer, kept between calls, through which sat_sample downloads the
// ordered keys: a device-to-host copy into pageable memory runs at a fraction of the
// link's rate.  One call uses it at a time; a concurrent call copies directly.  Growing it
// frees the old buffer (cudaFreeHost, which waits for the device).
struct PinnedStage {
    std::mutex mu;
    void* p = nullptr;
    size_t cap = 0;
};
PinnedStage g_stage;

// Key buffers of freed solution sets (at most two, 1 MiB to 256 MiB each), kept for the
// next sat_sample: a fresh buffer of several MB costs a page fault per page when the
// download first writes it.
struct KeyCache {
    std::mutex mu;
    std::vector<KeyBuffer> bufs;
};
KeyCache g_keys;
constexpr size_t KEY_CACHE_MIN = (size_t)1 << 20, KEY_CACHE_MAX = (size_t)1 << 28;

// A buffer of n words: the smallest cached one that holds them, else a new one with an
// eighth to spare (the next call's solution count differs a little).
KeyBuffer take_key_buffer(size_t n) {
    KeyBuffer out;
    {
        std::lock_guard<std::mutex> lk(g_keys.mu);
        int best = -1;
        for (int i = 0; i < (int)g_keys.bufs.size(); i++)
            if (g_keys.bufs[i].capacity() >= n && (best < 0 || g_keys.bufs[i].capacity() < g_keys.bufs[best].capacity()))
                best = i;
        if (best >= 0) {
            out = std::move(g_keys.bufs[best]);
            g_keys.bufs.erase(g_keys.bufs.begin() + best);
        }
    }
    if (out.capacity() < n) out.reserve(n + n / 8);
    out.resize(n);
    return out;
}

void give_key_buffer(KeyBuffer&& b) {
    const size_t bytes = b.capacity() * sizeof(uint32_t);
    if (bytes < KEY_CACHE_MIN || bytes > KEY_CACHE_MAX) return;
    std::lock_guard<std::mutex> lk(g_keys.mu);
    if (g_keys.bufs.size() >= 2) {  // keep the two largest
        auto small = std::min_element(g_keys.bufs.begin(), g_keys.bufs.end(),
                                      [](const KeyBuffer& x, const KeyBuffer& y) { return x.capacity() < y.capacity(); });
        if (small->capacity() >= b.capacity()) return;
        g_keys.bufs.erase(small);
    }
    g_keys.bufs.push_back(std::move(b));
}

// Device buffers of one call, stream-ordered (allocated and freed on the call's stream,
// from the library pool): freeing does not synchronise the device, so calls on other
// streams keep running.  An allocation the pool cannot serve is retried once after the
// pool's idle reserve is returned to the device.
struct Workspace {
    explicit Workspace(cudaStream_t s) : stream(s) {}
    cudaStream_t stream;
    std::vector<void*> bufs;
    float *V = nullptr, *m = nullptr, *v = nullptr, *adj = nullptr;
    void* act = nullptr;
    uint32_t *bits = nullptr, *keys = nullptr, *valid = nullptr;
    int64_t ldw = 0;
    const sat::DevAct* lay = nullptr;  // act layout of the fused steps
    ~Workspace() {
        for (void* b : bufs) cudaFreeAsync(b, stream);
    }
    bool alloc(void** p, size_t n) {
        if (n == 0) n = 16;
        cudaMemPool_t pool = nullptr;
        if (library_pool(&pool) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (cudaMallocFromPoolAsync(p, n, pool, stream) != cudaSuccess) {
            cudaGetLastError();
            cudaMemPoolTrimTo(pool, 0);
            if (cudaMallocFromPoolAsync(p, n, pool, stream) != cudaSuccess) {
                cudaGetLastError();
                return false;
            }
        }
        bufs.push_back(*p);
        return true;
    }
};

size_t act_bytes(int t) { return t == SAT_ACT_F32 ? 4 : 2; }

// NVTX ranges around a round and its phases, for profiler timelines (NVTX v3 is
// header-only: without an attached tool the calls do nothing).
struct NvtxPhases {
    bool open = false;
    explicit NvtxPhases(const char* round) { nvtxRangePushA(round); }
    void next(const char* phase) {
        if (open) nvtxRangePop();
        nvtxRangePushA(phase);
        open = true;
    }
    ~NvtxPhases() {
        if (open) nvtxRangePop();
        nvtxRangePop();
    }
};

size_t scratch_elems(int64_t rows, int64_t B) {
    return (size_t)((B + SAT_TILE_SAMPLES - 1) / SAT_TILE_SAMPLES) * (size_t)rows * SAT_TILE_SAMPLES;
}

}  // namespace

sat_status sat_cached_memory(uint64_t* reserved_bytes, uint64_t* used_bytes) {
    if (!reserved_bytes || !used_bytes) return fail(SAT_ERR_ARG, "NULL argument");
    cudaMemPool_t pool = nullptr;
    cudaError_t e = library_pool(&pool);
    uint64_t r = 0, u = 0;
    if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r);
    if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SAT_ERR_CUDA, std::string("memory pool: ") + cudaGetErrorString(e));
    }
    *reserved_bytes = r;
    *used_bytes = u;
    return SAT_OK;
}

sat_status sat_release_cached_memory(void) {
    {
        std::lock_guard<std::mutex> lk(g_stage.mu);
        if (g_stage.p) cudaFreeHost(g_stage.p);
        g_stage.p = nullptr;
        g_stage.cap = 0;
    }
    {
        std::lock_guard<std::mutex> lk(g_keys.mu);
        g_keys.bufs.clear();
    }
    sat::round_cache_clear();
    cudaMemPool_t pool = nullptr;
    cudaError_t e = library_pool(&pool);
    if (e == cudaSuccess) e = cudaMemPoolTrimTo(pool, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SAT_ERR_CUDA, std::string("memory pool: ") + cudaGetErrorString(e));
    }
    return SAT_OK;
}

// Early exit: epochs of check_every steps over the whole batch; after each, the
// valid samples are harvested into the dedup set and they (and samples older
// than max_age) restart from new starts drawn on the Philox stream of round
// first_round + 1 + epoch (or from the proposal network).
static sat_status sample_early_exit(const sat_plan* p, sat_dedup* d, const sat_sample_opts* o, uint64_t n_wanted,
                                    sat_sample_stats* st, Workspace& w, cudaStream_t str) {
    const sat::DevPlan& dp = p->dp;
    const int64_t B = o->batch;
    const size_t npi = (size_t)dp.n_pi;
    int32_t* age = nullptr;
    uint32_t* restart = nullptr;
    float* Vp = nullptr;
    if (!w.alloc((void**)&age, (size_t)B * 4) || !w.alloc((void**)&restart, (size_t)w.ldw * 4) ||
        (o->proposal && !w.alloc((void**)&Vp, npi * B * 4)))
        return fail(SAT_ERR_OOM, "cudaMalloc failed for the early-exit state");
    cudaEvent_t ev[5];
    for (auto& e : ev) CK(cudaEventCreate(&e));
    struct EvGuard {
        cudaEvent_t* e;
        ~EvGuard() { for (int i = 0; i < 5; i++) cudaEventDestroy(e[i]); }
    } guard{ev};
    sat_status s;
    const sat::OptParams op = opt_of(&o->opt);
    const int k = o->check_every;
    const int max_age = o->max_age > 0 ? o->max_age : std::max(1, o->steps);
    const int spl = o->steps_per_launch > 0 ? o->steps_per_launch : k;
    const int64_t budget = (int64_t)o->max_rounds * o->steps;
    sat_sample_stats acc{};
    std::vector<uint32_t> hvalid(w.ldw), hrestart(w.ldw);
    uint64_t have = 0;
    sat_status result = SAT_PARTIAL;
    // initial starts (round first_round)
    CK(cudaEventRecord(ev[0], str));
    if (o->init_logits) {
        CK(cudaMemcpy2DAsync(w.V, B * 4, o->init_logits, o->init_ld * 4, B * 4, npi, cudaMemcpyDeviceToDevice, str));
    } else if (o->proposal) {
        if ((s = sat_mlp_propose(o->proposal, o->seed, o->first_round, o->proposal_tau, w.V, B, B, o->stream)) !=
            SAT_OK)
            return s;
    } else {
        CK(sat::launch_init_normal(dp, o->seed, o->first_round, o->init_scale, w.V, B, B, str));
    }
    CK(cudaMemsetAsync(w.m, 0, npi * B * 4, str));
    CK(cudaMemsetAsync(w.v, 0, npi * B * 4, str));
    CK(cudaMemsetAsync(age, 0, (size_t)B * 4, str));
    CK(cudaEventRecord(ev[1], str));
    float ms0 = 0.0f;
    CK(cudaEventSynchronize(ev[1]));
    CK(cudaEventElapsedTime(&ms0, ev[0], ev[1]));
    acc.ms_init += ms0;
    acc.ms_total += ms0;
    acc.samples = (uint64_t)B;
    for (int64_t done = 0, e = 0; done < budget; e++) {
        const int kk = (int)std::min<int64_t>(k, budget - done);
        NvtxPhases ph("sat.epoch");
        ph.next("sat.steps");
        CK(cudaEventRecord(ev[0], str));
        for (int t0 = 1; t0 <= kk; t0 += spl)
            CK(sat::launch_steps(dp, *w.lay, o->act_dtype, op, w.V, w.m, w.v, B, w.act, w.adj, nullptr, t0,
                                 std::min(spl, kk - t0 + 1), B, str, age));
        CK(cudaEventRecord(ev[1], str));
        ph.next("sat.verify");
        CK(sat::launch_threshold(dp, w.V, B, w.bits, w.ldw, w.keys, B, str));
        CK(sat::launch_hard_eval(dp, w.bits, w.ldw, B, str));
        CK(sat::launch_cnf_check(dp, w.bits, w.ldw, w.valid, B, str));
        CK(cudaEventRecord(ev[2], str));
        ph.next("sat.dedup");
        uint64_t n = 0;
        if ((s = sat_dedup_count(d, &n, str)) != SAT_OK) return s;
        if (n + (uint64_t)B > d->d.pool_capacity) return fail(SAT_ERR_TABLE_FULL, "dedup table is full");
        CK(sat::launch_dedup_insert(d->d, w.keys, w.valid, B, nullptr, nullptr, d->slot_of, str));
        CK(cudaEventRecord(ev[3], str));
        ph.next("sat.restart");
        CK(sat::launch_retire(w.valid, age, restart, kk, max_age, B, str));
        const uint32_t round = o->first_round + 1u + (uint32_t)e;
        if (o->proposal && (s = sat_mlp_propose(o->proposal, o->seed, round, o->proposal_tau, Vp, B, B, o->stream)) !=
                               SAT_OK)
            return s;
        CK(sat::launch_restart(dp, restart, o->seed, round, o->init_scale, Vp, B, w.V, w.m, w.v, B, B, str));
        CK(cudaEventRecord(ev[4], str));
        CK(cudaMemcpyAsync(hvalid.data(), w.valid, w.ldw * 4, cudaMemcpyDeviceToHost, str));
        CK(cudaMemcpyAsync(hrestart.data(), restart, w.ldw * 4, cudaMemcpyDeviceToHost, str));
        unsigned int status = 0;
        CK(cudaMemcpyAsync(&status, d->d.status, sizeof(status), cudaMemcpyDeviceToHost, str));
        CK(cudaStreamSynchronize(str));
        if (status) return fail(SAT_ERR_TABLE_FULL, "dedup probe limit reached");
        uint32_t pst = 0;
        if ((s = sat_plan_status(p, &pst, 1, str)) != SAT_OK) return s;
        if (pst) return fail(SAT_ERR_CUDA, "a bounded wait in the step kernel expired (status " + std::to_string(pst) + ")");
        float ms[4];
        for (int i = 0; i < 4; i++) CK(cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]));
        acc.ms_steps += ms[0];
        acc.ms_verify += ms[1];
        acc.ms_dedup += ms[2];
        acc.ms_init += ms[3];
        acc.ms_total += ms[0] + ms[1] + ms[2] + ms[3];
        acc.rounds++;
        for (uint32_t x : hvalid) acc.valid += (uint64_t)__builtin_popcount(x);
        for (uint32_t x : hrestart) acc.samples += (uint64_t)__builtin_popcount(x);
        done += kk;
        if ((s = sat_dedup_count(d, &have, str)) != SAT_OK) return s;
        if (have >= n_wanted) {
            result = SAT_OK;
            break;
        }
    }
    acc.unique = have;
    if (st) *st = acc;
    if (result == SAT_PARTIAL) g_err = "budget ended before n_wanted distinct solutions";
    return result;
}

sat_status sat_sample_plan(const sat_plan* p, sat_dedup* d, const sat_sample_opts* o, uint64_t n_wanted,
                           sat_sample_stats* st) {
    if (!p || !d || !o) return fail(SAT_ERR_ARG, "NULL argument");
    const int64_t B = o->batch;
    if (B <= 0 || B > d->max_batch) return fail(SAT_ERR_ARG, "batch must be in 1..dedup max_batch");
    if (o->steps < 0 || o->max_rounds < 1 || !opt_ok(&o->opt)) return fail(SAT_ERR_ARG, "bad steps/rounds/optimiser");
    if (o->check_every < 0 || o->max_age < 0) return fail(SAT_ERR_ARG, "bad check_every / max_age");
    if (o->act_dtype < SAT_ACT_F32 || o->act_dtype > SAT_ACT_F16) return fail(SAT_ERR_ARG, "bad act_dtype");
    if (o->init_logits && o->init_ld < B) return fail(SAT_ERR_ARG, "init_ld < batch");
    if (o->recompute_segment < 0) return fail(SAT_ERR_ARG, "recompute_segment must be >= 0");
    sat_status s = check_device(p->device);
    if (s != SAT_OK) return s;
    cudaStream_t str = S(o->stream);
    const sat::DevPlan& dp = p->dp;
    Workspace w(str);
    if ((s = plan_layout(p, o->recompute_segment, &w.lay)) != SAT_OK) return s;
    w.ldw = (B + 31) / 32;
    const size_t npi = (size_t)dp.n_pi;
    if (!w.alloc((void**)&w.V, npi * B * 4) || !w.alloc((void**)&w.m, npi * B * 4) ||
        !w.alloc((void**)&w.v, npi * B * 4) ||
        !w.alloc(&w.act, scratch_elems(w.lay->n_act_rows, B) * act_bytes(o->act_dtype)) ||
        !w.alloc((void**)&w.adj, scratch_elems(dp.n_adj_rows, B) * 4) ||
        !w.alloc((void**)&w.bits, (size_t)dp.n_nodes * w.ldw * 4) ||
        !w.alloc((void**)&w.keys, (size_t)B * std::max(1, dp.key_words) * 4) ||
        !w.alloc((void**)&w.valid, (size_t)w.ldw * 4))
        return fail(SAT_ERR_OOM, "cudaMalloc failed for the sampling workspace");
    if (o->check_every > 0) return sample_early_exit(p, d, o, n_wanted, st, w, str);
    cudaEvent_t ev[5];
    for (auto& e : ev) CK(cudaEventCreate(&e));
    struct EvGuard {
        cudaEvent_t* e;
        ~EvGuard() { for (int i = 0; i < 5; i++) cudaEventDestroy(e[i]); }
    } guard{ev};
    sat_sample_stats acc{};
    const sat::OptParams op = opt_of(&o->opt);
    const int spl = o->steps_per_launch > 0 ? o->steps_per_launch : std::max(1, o->steps);
    // Plain GD on FP32 activations: the whole round (init, steps, threshold, Boolean pass,
    // clause check) in the plan's instance-compiled kernel when it keeps every value in
    // registers.
    bool use_round = false;
    if (p->round && p->dp.step_kernel == SAT_STEP_KERNEL_AUTO && o->opt.optimizer == SAT_OPT_GD &&
        o->act_dtype == SAT_ACT_F32 && !o->proposal && !o->init_logits) {
        std::string err;
        if (p->round->ensure(err) != cudaSuccess) return fail(SAT_ERR_CUDA, err);
        use_round = p->round->mod->spill_bytes == 0;
    }
    std::vector<uint32_t> hvalid(w.ldw);
    uint64_t have = 0;
    sat_status result = SAT_PARTIAL;
    for (int r = 0; r < o->max_rounds; r++) {
        NvtxPhases ph("sat.round");
        if (use_round) {
            ph.next("sat.round_kernel");
            CK(cudaEventRecord(ev[0], str));
            CK(cudaEventRecord(ev[1], str));
            CK(p->round->launch(o->seed, o->first_round + (uint32_t)r, o->init_scale, op.lr, o->steps, nullptr, 0,
                                w.keys, w.valid, B, str));
            CK(cudaEventRecord(ev[2], str));
            CK(cudaEventRecord(ev[3], str));
        } else {
            ph.next("sat.init");
            CK(cudaEventRecord(ev[0], str));
            if (r == 0 && o->init_logits) {
                CK(cudaMemcpy2DAsync(w.V, B * 4, o->init_logits, o->init_ld * 4, B * 4, npi, cudaMemcpyDeviceToDevice,
                                     str));
            } else if (o->proposal) {
                if ((s = sat_mlp_propose(o->proposal, o->seed, o->first_round + (uint32_t)r, o->proposal_tau, w.V, B, B,
                                         o->stream)) != SAT_OK)
                    return s;
            } else {
                CK(sat::launch_init_normal(dp, o->seed, o->first_round + (uint32_t)r, o->init_scale, w.V, B, B, str));
            }
            if (o->opt.optimizer == SAT_OPT_ADAM) {  // GD neither reads nor writes m, v
                CK(cudaMemsetAsync(w.m, 0, npi * B * 4, str));
                CK(cudaMemsetAsync(w.v, 0, npi * B * 4, str));
            }
            CK(cudaEventRecord(ev[1], str));
            ph.next("sat.steps");
            for (int t0 = 1; t0 <= o->steps; t0 += spl)
                CK(sat::launch_steps(dp, *w.lay, o->act_dtype, op, w.V, w.m, w.v, B, w.act, w.adj, nullptr, t0,
                                     std::min(spl, o->steps - t0 + 1), B, str));
            CK(cudaEventRecord(ev[2], str));
            ph.next("sat.verify");
            CK(sat::launch_threshold(dp, w.V, B, w.bits, w.ldw, w.keys, B, str));
            CK(sat::launch_hard_eval(dp, w.bits, w.ldw, B, str));
            CK(sat::launch_cnf_check(dp, w.bits, w.ldw, w.valid, B, str));
            CK(cudaEventRecord(ev[3], str));
        }
        ph.next("sat.dedup");
        uint64_t n = 0;
        if ((s = sat_dedup_count(d, &n, str)) != SAT_OK) return s;
        if (n + (uint64_t)B > d->d.pool_capacity) return fail(SAT_ERR_TABLE_FULL, "dedup table is full");
        CK(sat::launch_dedup_insert(d->d, w.keys, w.valid, B, nullptr, nullptr, d->slot_of, str));
        CK(cudaEventRecord(ev[4], str));
        CK(cudaMemcpyAsync(hvalid.data(), w.valid, w.ldw * 4, cudaMemcpyDeviceToHost, str));
        unsigned int status = 0;
        CK(cudaMemcpyAsync(&status, d->d.status, sizeof(status), cudaMemcpyDeviceToHost, str));
        CK(cudaStreamSynchronize(str));
        if (status) return fail(SAT_ERR_TABLE_FULL, "dedup probe limit reached");
        uint32_t pst = 0;
        if ((s = sat_plan_status(p, &pst, 1, str)) != SAT_OK) return s;
        if (pst) return fail(SAT_ERR_CUDA, "a bounded wait in the step kernel expired (status " + std::to_string(pst) + ")");
        float ms[4];
        for (int i = 0; i < 4; i++) CK(cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]));
        acc.ms_init += ms[0];
        acc.ms_steps += ms[1];
        acc.ms_verify += ms[2];
        acc.ms_dedup += ms[3];
        acc.ms_total += ms[0] + ms[1] + ms[2] + ms[3];
        acc.rounds++;
        acc.samples += (uint64_t)B;
        for (uint32_t x : hvalid) acc.valid += (uint64_t)__builtin_popcount(x);
        if ((s = sat_dedup_count(d, &have, str)) != SAT_OK) return s;
        if (have >= n_wanted) {
            result = SAT_OK;
            break;
        }
    }
    acc.unique = have;
    if (st) *st = acc;
    if (result == SAT_PARTIAL) g_err = "budget ended before n_wanted distinct solutions";
    return result;
}

sat_status sat_sample(const sat_circuit* c, const sat_cnf* cnf, const sat_sample_opts* o, uint64_t n_wanted,
                      sat_solutions** out, sat_sample_stats* st) {
    if (!c || !cnf || !o || !out) return fail(SAT_ERR_ARG, "NULL argument");
    *out = nullptr;
    auto t0 = std::chrono::steady_clock::now();
    sat_plan* p = nullptr;
    sat_status s = sat_plan_create(c, cnf, &p);
    if (s != SAT_OK) return s;
    if (o->step_kernel != SAT_STEP_KERNEL_AUTO && (s = sat_plan_set_step_kernel(p, o->step_kernel)) != SAT_OK) {
        sat_plan_free(p);
        return s;
    }
    struct PG {
        sat_plan* p;
        sat_dedup* d = nullptr;
        ~PG() { sat_dedup_free(d); sat_plan_free(p); }
    } pg{p};
    // Early exit can harvest more than one solution per slot and round: room for
    // n_wanted (capped by the budget's sample-epochs) plus one batch.
    uint64_t max_keys = (uint64_t)o->batch * (uint64_t)std::max(1, o->max_rounds);
    if (o->check_every > 0) {
        const uint64_t epochs = ((uint64_t)std::max(1, o->max_rounds) * (uint64_t)std::max(0, o->steps) +
                                 (uint64_t)o->check_every - 1) / (uint64_t)o->check_every;
        max_keys = std::min<uint64_t>(n_wanted, (uint64_t)o->batch * std::max<uint64_t>(1, epochs)) +
                   (uint64_t)o->batch;
    }
    if ((s = sat_dedup_create(p, max_keys, o->batch, &pg.d)) != SAT_OK) return s;
    auto t1 = std::chrono::steady_clock::now();
    sat_sample_stats acc{};
    sat_status r = sat_sample_plan(p, pg.d, o, n_wanted, &acc);
    if (r != SAT_OK && r != SAT_PARTIAL) return r;
    std::string partial_msg = g_err;
    auto t2 = std::chrono::steady_clock::now();
    auto* sol = new sat_solutions();
    sol->n_vars = p->info.n_vars;
    sol->n_pi = p->info.n_pi;
    sol->key_words = p->info.key_words;
    sol->count = acc.unique;
    // canonical order: ascending packed input vector (highest word most significant), sorted
    // on the device by the top 64 bits; keys that share them are ordered here
    const uint32_t kw = sol->key_words;
    sol->keys = take_key_buffer(sol->count * kw);
    if (sol->count > 0 && kw > 0) {
        Workspace ow(S(o->stream));
        uint64_t* hi = nullptr;
        uint32_t *idx = nullptr, *sorted = nullptr;
        const uint64_t n2 = sat::key_order_pad(sol->count);
        if (!ow.alloc((void**)&hi, n2 * 8) || !ow.alloc((void**)&idx, n2 * 4) ||
            !ow.alloc((void**)&sorted, sol->count * kw * 4)) {
            delete sol;
            return fail(SAT_ERR_OOM, "cudaMalloc failed for the solution order");
        }
        const size_t bytes = sol->count * kw * 4;
        std::unique_lock<std::mutex> lk(g_stage.mu, std::try_to_lock);
        if (lk.owns_lock() && g_stage.cap < bytes) {
            if (g_stage.p) cudaFreeHost(g_stage.p);
            g_stage.p = nullptr;
            g_stage.cap = 0;
            size_t want = (size_t)1 << 20;  // powers of two from 1 MiB: few regrowths
            while (want < bytes) want <<= 1;
            if (cudaMallocHost(&g_stage.p, want) == cudaSuccess)
                g_stage.cap = want;
            else
                cudaGetLastError();
        }
        void* dst = lk.owns_lock() && g_stage.cap >= bytes ? g_stage.p : (void*)sol->keys.data();
        cudaError_t e = sat::launch_key_order(pg.d->d.pool, (int)kw, sol->count, hi, idx, sorted, S(o->stream));
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, sorted, bytes, cudaMemcpyDeviceToHost, S(o->stream));
        if (e == cudaSuccess) e = cudaStreamSynchronize(S(o->stream));
        if (e == cudaSuccess && dst != (void*)sol->keys.data()) std::memcpy(sol->keys.data(), dst, bytes);
        if (lk.owns_lock()) lk.unlock();
        if (e != cudaSuccess) {
            delete sol;
            return fail(SAT_ERR_CUDA, std::string("solution order: ") + cudaGetErrorString(e));
        }
        if (kw > 2) {  // runs with equal top 64 bits: full-key order
            auto row = [&](uint64_t i) { return sol->keys.data() + i * kw; };
            for (uint64_t a = 0; a < sol->count;) {
                uint64_t b = a + 1;
                while (b < sol->count && row(b)[kw - 1] == row(a)[kw - 1] && row(b)[kw - 2] == row(a)[kw - 2]) b++;
                if (b - a > 1) {
                    std::vector<std::vector<uint32_t>> run;
                    for (uint64_t i = a; i < b; i++) run.emplace_back(row(i), row(i) + kw);
                    std::sort(run.begin(), run.end(), [&](const std::vector<uint32_t>& x, const std::vector<uint32_t>& y) {
                        return std::lexicographical_compare(x.rbegin(), x.rend(), y.rbegin(), y.rend());
                    });
                    for (uint64_t i = a; i < b; i++) std::copy(run[i - a].begin(), run[i - a].end(), row(i));
                }
                a = b;
            }
        }
    }
    sol->f_in0 = p->f_in0;
    sol->f_in1 = p->f_in1;
    sol->f_gop = p->f_gop;
    sol->var_full = p->var_full;
    sol->var_neg = p->var_neg;
    auto t3 = std::chrono::steady_clock::now();
    acc.ms_upload = std::chrono::duration<double, std::milli>(t1 - t0).count();
    acc.ms_download = std::chrono::duration<double, std::milli>(t3 - t2).count();
    if (st) *st = acc;
    *out = sol;
    if (r == SAT_PARTIAL) g_err = partial_msg;
    return r;
}

uint64_t sat_solutions_count(const sat_solutions* s) { return s ? s->count : 0; }
uint32_t sat_solutions_nvars(const sat_solutions* s) { return s ? s->n_vars : 0; }

sat_status sat_solutions_copy(const sat_solutions* s, uint64_t first, uint64_t count, uint64_t* words_out) {
    if (!s || (count && !words_out)) return fail(SAT_ERR_ARG, "NULL argument");
    if (first + count > s->count) return fail(SAT_ERR_ARG, "range beyond the solution count");
    const uint64_t nw = (s->n_vars + 63) / 64;
    std::fill(words_out, words_out + count * nw, 0ull);
    const size_t n_nodes = s->n_pi + s->f_in0.size();
    std::vector<uint64_t> node(n_nodes);
    // 64 solutions at a time: bit j of each node word = solution (base + j)
    for (uint64_t base = 0; base < count; base += 64) {
        const uint64_t nb = std::min<uint64_t>(64, count - base);
        std::fill(node.begin(), node.end(), 0ull);
        for (uint64_t j = 0; j < nb; j++) {
            const uint32_t* key = &s->keys[(first + base + j) * s->key_words];
            for (uint32_t i = 0; i < s->n_pi; i++)
                if ((key[i >> 5] >> (i & 31)) & 1u) node[i] |= 1ull << j;
        }
        for (size_t g = 0; g < s->f_in0.size(); g++) {
            uint64_t a = node[s->f_in0[g]], b = node[s->f_in1[g]];
            const uint8_t f = s->f_gop[g];
            if (f & 4) a = ~a;
            if (f & 8) b = ~b;
            const uint8_t op = f & 3;
            node[s->n_pi + g] = op == 0 ? (a & b) : op == 1 ? (a | b) : (a ^ b);
        }
        for (uint32_t v = 1; v <= s->n_vars; v++) {
            uint64_t x = node[s->var_full[v]];
            if (s->var_neg[v]) x = ~x;
            const uint64_t wi = (v - 1) >> 6, bi = (v - 1) & 63;
            for (uint64_t j = 0; j < nb; j++)
                if ((x >> j) & 1ull) words_out[(base + j) * nw + wi] |= 1ull << bi;
        }
    }
    return SAT_OK;
}

void sat_solutions_free(sat_solutions* s) {
    if (!s) return;
    give_key_buffer(std::move(s->keys));
    delete s;
}

}  // extern "C"
