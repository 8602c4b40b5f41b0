// Device-side plan and kernel launchers (internal; the C ABI wraps these).
#pragma once
#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <mutex>

#define SAT_TILE_SAMPLES 128  // samples per scratch tile (SAT_TILE in the C ABI)

namespace sat {

// Activation layout of a tile's act scratch.  k = 0: every cone node has its own row
// (row = node).  k > 0 (level-segment recomputation): levels 1.. are cut into segments
// of k levels; a level is kept ("stored") when it is among the top max_span levels of
// its segment (the inputs the next segment's gates read) or holds an output; the other
// levels of segment j share scratch buffer j % 2 and are evaluated again in the
// backward pass.  Level 0 is always kept.
struct DevAct {
    int32_t k = 0;
    int64_t n_act_rows = 0;            // rows of one tile's act scratch
    const int32_t* act_off = nullptr;  // [n_clev + 1]: act row of the first node of level l
    const uint8_t* stored = nullptr;   // [n_clev + 1]: 1 = kept level (k > 0 only)
    const int2* gate = nullptr;        // per cone gate: (act row of in0 | gop << 28, act row of in1)
    const int4* edge = nullptr;        // fan-out edges with the sibling's act row
    const int32_t* out_row = nullptr;  // act rows of the outputs
};

// Device copy of a Plan.  All pointers are device pointers owned by the plan.
struct DevPlan {
    // cone schedule (gradient loop)
    int32_t n_cone_pi = 0;
    int64_t n_cone = 0;
    int32_t n_clev = 0;                 // cone levels 1..n_clev
    int32_t max_span = 0;               // max level distance of a cone edge (consumer level - input level)
    const int32_t* c_level_off = nullptr;
    const int2* c_gate = nullptr;       // per cone gate: (in0 | gop << 28, in1)
    const int32_t* cone_pi_row = nullptr;
    const int32_t* fo_off = nullptr;    // [n_cone + 1]
    const int4* fo_edge = nullptr;      // (consumer's adj row (seed_row for seeds), sibling | last << 31, c0 bits, c1 bits)
    // Adjoint scratch rows of a tile: level 0 (the cone inputs) in rows [0, n_cone_pi); a
    // gate level l is live only until the backward pass has finished level l - max_span, so
    // with adj_slots > 0 level l >= 1 occupies slot (l - 1) % adj_slots of a ring of
    // adj_slots = max_span + 1 slots of adj_slot_rows rows each (adj_slots = 0: row = node).
    int64_t n_adj_rows = 0;
    int32_t adj_slots = 0, adj_slot_rows = 0;
    int32_t seed_row = 0;               // last adj row: the output seeds' scale (the consumer row of seed edges)
    int32_t n_out = 0;
    const int32_t* c_out_node = nullptr;
    const float* out_target = nullptr;
    // full schedule (Boolean pass)
    int32_t n_pi = 0;
    int64_t n_nodes = 0;
    int32_t n_flev = 0;
    const int32_t* f_level_off = nullptr;
    const int2* f_gate = nullptr;       // per gate: (in0 | gop << 28, in1)
    // CNF in node space
    int64_t n_clauses = 0;
    const int64_t* cl_off = nullptr;
    const int32_t* cl_lit = nullptr;    // node << 1 | negation
    int32_t key_words = 0;              // ceil(n_pi / 32)
    unsigned int* status = nullptr;     // device status word (bit 2: an async-copy wait expired)
    // Adjoint ring rows that no backward level below l reads (their consumer's inputs all lie
    // at levels >= l) and whose slot the next level does not reuse: rows
    // dead_row[dead_off[l] .. dead_off[l + 1]) are dropped from L2 after level l (ring only).
    const int32_t* dead_off = nullptr;  // [n_clev + 2]
    const int32_t* dead_row = nullptr;
    // Node runs of the adjoint balanced by fan-out edges (a warp's adjoint work is its edges,
    // and fan-outs vary from node to node): for the k-th warp count W = adj_run_w[k] of the
    // step kernels (warps serving one tile), adj_run[adj_run_base[k] + l * (W + 1) + w] is
    // the first cone node of warp w's run at level l (w = W: the level's end).  A warp count
    // without a table splits each level's nodes evenly.
    static constexpr int ADJ_RUN_SETS = 4;
    int32_t adj_run_w[ADJ_RUN_SETS] = {};
    int64_t adj_run_base[ADJ_RUN_SETS] = {};
    const int32_t* adj_run = nullptr;
    DevAct full;                        // the full act layout (row = node)
    int32_t step_kernel = 0;            // fused steps: STEP_KERNEL_AUTO / _TILED / _RESIDENT
    // host mirrors of the level offsets (launch loops need them)
    const int32_t* h_c_level_off = nullptr;
    const int32_t* h_f_level_off = nullptr;
};

// Adjoint row of the first node of level l >= 1.
inline __host__ __device__ int64_t adj_level_row(const DevPlan& p, int l, int32_t level_off) {
    return p.adj_slots ? (int64_t)p.n_cone_pi + (int64_t)((l - 1) % p.adj_slots) * p.adj_slot_rows
                       : (int64_t)level_off;
}

enum ActType { ACT_F32 = 0, ACT_BF16 = 1, ACT_F16 = 2 };

// Warps that serve one tile in the tiled step kernels (FP32 and 16-bit activations, one CTA
// and 2-CTA clusters): the warp counts DevPlan::adj_run is built for.
void step_warp_counts(int32_t out[DevPlan::ADJ_RUN_SETS]);

// A set-up step that must run once on every device: attributes set with
// cudaFuncSetAttribute (the dynamic shared-memory opt-in) hold for the device that was
// current when they were set, so a plan on a second GPU needs them set there too.
// run(f) calls f() the first time it is called with a given device current and
// returns that result on every later call with the same device current.
class PerDeviceOnce {
  public:
    template <typename F>
    cudaError_t run(F&& f) {
        int dev = -1;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
        if (done_[dev].load(std::memory_order_acquire)) return result_[dev];
        std::lock_guard<std::mutex> lock(mu_);
        if (!done_[dev].load(std::memory_order_relaxed)) {
            result_[dev] = f();
            done_[dev].store(true, std::memory_order_release);
        }
        return result_[dev];
    }

  private:
    static constexpr int kMaxDevices = 64;
    std::mutex mu_;
    std::atomic<bool> done_[kMaxDevices] = {};
    cudaError_t result_[kMaxDevices] = {};
};

// Kernel of the fused steps: AUTO takes the shared-memory resident kernel when the
// plan's per-sample state fits (resident_config), else the tiled one.
enum StepKernel { STEP_KERNEL_AUTO = 0, STEP_KERNEL_TILED = 1, STEP_KERNEL_RESIDENT = 2 };
constexpr size_t RESIDENT_SMEM_MAX = 200u * 1024u;  // dynamic shared memory of one resident CTA

struct OptParams {
    int opt = 0;  // 0 Adam, 1 GD
    float lr = 0.1f, b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
};

// Kernel launchers; return cudaSuccess or the launch error.
cudaError_t launch_init_normal(const DevPlan& p, uint64_t seed, uint32_t round, float scale,
                               float* V, int64_t ldv, int64_t B, cudaStream_t s);
// act / adj scratch is tile-major: tile t (samples 128t .. 128t+127) owns rows
// [n_act_rows][128] of act starting at element t * n_act_rows * 128 (SAT_TILE = 128),
// and [n_adj_rows][128] of adj likewise.  forward / backward use the full act layout.
cudaError_t launch_forward(const DevPlan& p, int act_type, const float* V, int64_t ldv, void* act, float* loss,
                           int64_t B, cudaStream_t s);
cudaError_t launch_backward(const DevPlan& p, int act_type, const float* V, int64_t ldv, const void* act, float* adj,
                            const float* grad_loss, float* gV, int64_t B, cudaStream_t s);
// Adam step of sample b at in-launch step s: t0 + s, plus age[b] when age is given.
// lay: the act layout (the full one, or a recomputation layout of the plan).
cudaError_t launch_steps(const DevPlan& p, const DevAct& lay, int act_type, const OptParams& o, float* V, float* m,
                         float* v, int64_t ldv, void* act, float* adj, float* loss, int t0, int n_steps, int64_t B,
                         cudaStream_t s, const int32_t* age = nullptr);
// The shared-memory resident kernel of the fused steps (32 samples per CTA): whether the
// plan fits it with activations of act_type, its warps per CTA and dynamic shared memory.
bool resident_config(const DevPlan& p, int act_type, int* warps, size_t* smem);
// Whether launch_steps runs the resident kernel for this plan and act_type (AUTO and the
// plan fits it, or RESIDENT); the tiled kernel otherwise, which uses the act/adj scratch.
bool steps_use_resident(const DevPlan& p, int act_type);
cudaError_t launch_steps_resident(const DevPlan& p, int act_type, const OptParams& o, float* V, float* m, float* v,
                                  int64_t ldv, float* loss, int t0, int n_steps, int64_t B, cudaStream_t s,
                                  const int32_t* age = nullptr);
// Early exit: restart[b] = valid(b) or age[b] + k >= max_age (bit-packed like valid);
// age[b] = 0 where restarting, else age[b] + k.
cudaError_t launch_retire(const uint32_t* valid, int32_t* age, uint32_t* restart, int k, int max_age, int64_t B,
                          cudaStream_t s);
// Restarted samples get a new start: V[:, b] = src[:, b] (src non-null) or scale * N(0, 1)
// from the init stream of `round` (the values launch_init_normal would draw); m = v = 0.
cudaError_t launch_restart(const DevPlan& p, const uint32_t* restart, uint64_t seed, uint32_t round, float scale,
                           const float* src, int64_t lds, float* V, float* m, float* v, int64_t ldv, int64_t B,
                           cudaStream_t s);
// Diagnostic: a bounded wait (limit_ns) on an mbarrier nothing completes; sets bit 2 of *status.
cudaError_t launch_bounded_wait_diag(unsigned* status, uint64_t limit_ns, cudaStream_t s);
cudaError_t launch_opt_update(const DevPlan& p, const OptParams& o, float* V, float* m, float* v,
                              const float* gV, int64_t ldv, int t, int64_t B, cudaStream_t s);
cudaError_t launch_threshold(const DevPlan& p, const float* V, int64_t ldv, uint32_t* node_bits,
                             int64_t ldw, uint32_t* keys, int64_t B, cudaStream_t s);
cudaError_t launch_hard_eval(const DevPlan& p, uint32_t* node_bits, int64_t ldw, int64_t B, cudaStream_t s);
cudaError_t launch_cnf_check(const DevPlan& p, const uint32_t* node_bits, int64_t ldw, uint32_t* valid,
                             int64_t B, cudaStream_t s);

// Device hash set of distinct solutions (keys = packed primary-input bits).
struct DevDedup {
    int32_t key_words = 0;
    uint64_t capacity = 0;            // slots (power of two)
    uint64_t pool_capacity = 0;       // keys that can be stored
    unsigned long long* slots = nullptr;
    uint32_t* pool = nullptr;         // [pool_capacity][key_words]
    unsigned long long* count = nullptr;   // device counter of stored keys
    unsigned int* status = nullptr;        // bit 0: table full / probe limit hit
    uint32_t max_probe = 0;
};

cudaError_t launch_dedup_clear(DevDedup& d, cudaStream_t s);

// Canonical order of n keys (kw uint32 words each, the highest word most significant):
// out[j] = keys[order[j]], ascending by the top 64 bits, ties by position (full-key order
// within a tie is left to the caller).  Scratch: hi, idx of key_order_pad(n) entries.
uint64_t key_order_pad(uint64_t n);
cudaError_t launch_key_order(const uint32_t* keys, int kw, uint64_t n, uint64_t* hi, uint32_t* idx, uint32_t* out,
                             cudaStream_t s);
// slot_of: scratch [B] (slot taken by each sample, or ~0).
cudaError_t launch_dedup_insert(DevDedup& d, const uint32_t* keys, const uint32_t* valid, int64_t B,
                                unsigned long long* hashes, uint8_t* is_new, unsigned long long* slot_of,
                                cudaStream_t s);

}  // namespace sat
