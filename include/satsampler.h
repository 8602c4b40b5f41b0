/*
 * satsampler.h — C ABI of a GPU SAT sampler built on gradient descent over a
 * relaxed multi-level circuit (Ardakani, Kang, He, Huang, Wawrzynek,
 * "High-Throughput SAT Sampling", arXiv 2502.08673).
 *
 * Pipeline (Section III): a CNF (Section II-A) is transformed once on the host
 * into a multi-level, multi-output circuit (Algorithm 1 and its fallback); a
 * batch of b samples of primary-input logits V is embedded as P = sigmoid(V)
 * (Eq. 5), pushed through the relaxed circuit (Table 1, Eq. 6), scored by the
 * l2 loss on the constrained outputs (Eq. 7) and updated by gradient steps
 * (Eqs. 8-9, or Adam); the thresholded assignments that satisfy the original
 * CNF are kept, without duplicates (end of Section III-A).
 *
 * Conventions (all calls):
 *  - Every call returns sat_status; no C++ exception crosses this boundary.
 *    On failure sat_last_error() (thread-local) describes the cause.
 *  - Objects returned through an `out` pointer are owned by the caller and
 *    released by the matching *_free, which accepts NULL.  A plan, dedup set or
 *    network holds device memory: free it only after the work queued on it has
 *    finished (synchronise its streams first; *_free does not wait).
 *  - Inputs are never modified.  "Device" pointers are CUDA global-memory
 *    pointers on the current device; "host" pointers are ordinary memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Device calls are asynchronous on that stream unless stated otherwise.
 *  - Per-sample device arrays are node-major with the batch contiguous: row r
 *    of an array with leading dimension ld starts at element r * ld.
 *    V, m, v, gV: [n_pi][ldv] float32, ldv >= B, row r = primary input r in
 *    ascending DIMACS-variable order (sat_plan_pi_vars).  Bit arrays:
 *    [rows][ldw] uint32, ldw >= ceil(B/32), bit j of word w = sample 32 w + j.
 *  - Per-node scratch (act, adj) is tile-major: samples are grouped in tiles
 *    of SAT_TILE, and tile t owns the contiguous block [rows][SAT_TILE] that
 *    starts at element t * rows * SAT_TILE, so an array holds
 *    ceil(B/SAT_TILE) * rows * SAT_TILE elements.  act: rows = n_cone (row =
 *    cone node) or, under recomputation, the rows of that layout; adj: the input
 *    level, a ring of max_span + 1 gate levels and one row of seed scales
 *    (sat_plan_layout_elems gives both; sat_plan_scratch_elems is enough for
 *    either array without recomputation).  The padding samples of the last tile are written
 *    too.  act holds act_dtype elements, adj float32; both must be 16-byte
 *    aligned.
 *  - Deterministic for a given (seed, options, GPU).
 */
#ifndef SATSAMPLER_H
#define SATSAMPLER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SAT_ABI_VERSION 1
#define SAT_TILE 128  /* samples per scratch tile (one CTA of the step kernels) */

typedef enum sat_status {
    SAT_OK = 0,
    SAT_PARTIAL = 1,            /* sat_sample: budget spent before n_wanted distinct solutions */
    SAT_ERR_PARSE = -1,         /* malformed DIMACS */
    SAT_ERR_ARG = -2,           /* invalid argument (NULL, size, layout, alignment) */
    SAT_ERR_OOM = -3,           /* host or device allocation failed */
    SAT_ERR_CUDA = -4,          /* CUDA runtime error (message in sat_last_error) */
    SAT_ERR_TABLE_FULL = -5,    /* dedup table full, or probe limit hit */
    SAT_ERR_UNSAT_TRIVIAL = -6  /* the CNF holds an empty clause */
} sat_status;

typedef enum sat_act_dtype { SAT_ACT_F32 = 0, SAT_ACT_BF16 = 1, SAT_ACT_F16 = 2 } sat_act_dtype;
typedef enum sat_optimizer { SAT_OPT_ADAM = 0, SAT_OPT_GD = 1 } sat_optimizer;

typedef struct sat_cnf sat_cnf;
typedef struct sat_circuit sat_circuit;
typedef struct sat_plan sat_plan;
typedef struct sat_dedup sat_dedup;
typedef struct sat_solutions sat_solutions;
typedef struct sat_mlp sat_mlp;

/* Library version string and the last error of the calling thread. */
const char* sat_version(void);
const char* sat_last_error(void);

/* ----------------------------------------------------------------- CNF ---
 * DIMACS text (the format of Fig. 1(a)): `p cnf V C` header, `c` comment
 * lines, clauses of non-zero literals ended by 0 (may span lines), optional
 * `%` end marker.  A clause count different from C, a literal outside 1..V or
 * an unterminated clause is SAT_ERR_PARSE.  The library keeps its own copy of
 * `buf` (len bytes, need not be NUL-terminated). */
sat_status sat_cnf_from_dimacs(const char* buf, size_t len, sat_cnf** out);
sat_status sat_cnf_from_file(const char* path, sat_cnf** out);
sat_status sat_cnf_info(const sat_cnf* cnf, uint32_t* n_vars, uint64_t* n_clauses, uint64_t* n_lits);
void sat_cnf_free(sat_cnf* cnf);

/* ------------------------------------------------------ transformation ---
 * Algorithm 1 (Section III-A) with the fallback for under-specified clauses,
 * on the host.  A sub-clause window SC is grown clause by clause; a variable v
 * of SC is defined as f when f (from the clauses holding -v) is the complement
 * of the expression from the clauses holding v.  Defined variables become
 * intermediate, the other variables of the defining clauses primary inputs;
 * constant definitions and leftover clauses become outputs constrained to 1.
 * max_support (1..8, default 8) bounds the window's variables, max_window
 * (default 16) its clauses.  NULL opts = defaults.  SAT_ERR_UNSAT_TRIVIAL for
 * an empty clause. */
typedef struct sat_build_opts {
    uint32_t max_support;
    uint32_t max_window;
    uint32_t direct;   /* nonzero: no factorization, every (cleaned) clause is an OR output
                          constrained to 1 and every variable a primary input (the CNF side of
                          the paper's Fig. 5 comparison, for the direct-relaxation ablation) */
    uint32_t reorder;  /* nonzero: before Algorithm 1, sort the clauses by (largest variable,
                          longer first, position) so that the clauses defining a variable are
                          adjacent, ahead of unit clauses on it, even when the file interleaves
                          them; 0 = the file's order, as in the paper */
} sat_build_opts;

typedef struct sat_build_stats {
    uint32_t n_vars, n_pi, n_iv, n_outputs, n_const;
    uint64_t n_gates;          /* lowered 2-input gates, whole circuit */
    uint32_t n_cone_pi;        /* primary inputs in the outputs' fan-in cone */
    uint64_t n_cone_gates;     /* gates the gradient loop evaluates */
    uint32_t n_levels, n_cone_levels, max_span;
    uint64_t ops_cnf;          /* 2-input gate equivalents of the CNF (Fig. 5, middle) */
    uint64_t ops_circuit;      /* 2-input gate equivalents of the circuit */
    double transform_ms, plan_ms;
} sat_build_stats;

sat_status sat_circuit_build(const sat_cnf* cnf, const sat_build_opts* opts, sat_circuit** out,
                             sat_build_stats* stats /* nullable */);
/* Canonical text form of the transformation result: `vars N`, `pi ...`,
 * `def VAR KIND OUTNEG : lits` (SOP terms separated by ` |`), `out lits`.
 * Writes at most cap bytes (NUL-terminated when it fits); *len = full length. */
sat_status sat_circuit_dump(const sat_circuit* c, char* buf, size_t cap, size_t* len);
void sat_circuit_free(sat_circuit* c);

/* --------------------------------------------------------- device plan ---
 * Uploads the lowered circuit (2-input gates in level order, fan-out lists for
 * the adjoint) and the CNF (for the exact check) to the current device. */
typedef struct sat_plan_info {
    uint32_t n_vars, n_pi, n_cone_pi, n_outputs, n_cone_levels, n_levels, key_words, max_span;
    uint64_t n_cone;           /* cone inputs + cone gates: rows of the full act layout */
    uint64_t n_nodes;          /* rows of the Boolean node array: inputs + all gates */
    uint64_t n_cone_gates, n_gates, n_clauses, n_fanout_edges;
    uint64_t upload_bytes;     /* bytes copied host -> device by sat_plan_create */
} sat_plan_info;

sat_status sat_plan_create(const sat_circuit* c, const sat_cnf* cnf, sat_plan** out);
sat_status sat_plan_get_info(const sat_plan* p, sat_plan_info* info);
/* Host arrays: vars[n_pi] = DIMACS variable of V row r. */
sat_status sat_plan_pi_vars(const sat_plan* p, uint32_t* vars);
/* Host arrays per DIMACS variable v (index 0 unused, n_vars + 1 entries):
 * cone_node[v] = act row holding v's node (-1 outside the cone),
 * full_node[v] = row of the Boolean node array, neg[v] = 1 when v is the
 * complement of that node. */
sat_status sat_plan_var_nodes(const sat_plan* p, int64_t* cone_node, int64_t* full_node, uint8_t* neg);
/* Device status word of the plan's kernels (synchronises `stream`): 0 when
 * healthy; bit 2 = a bounded wait for an asynchronous copy expired, and the
 * results of that launch are invalid.  clear != 0 resets it. */
sat_status sat_plan_status(const sat_plan* p, uint32_t* status, int32_t clear, void* stream);
/* Diagnostic of the failure path of every asynchronous-copy wait in the step
 * kernels (which give up after 1 s): one warp polls, with the same bounded
 * wait but a bound of limit_us microseconds (1 .. 10^7), an mbarrier whose
 * phase no copy completes, and sets bit 2 (the plan status bit of an expired
 * wait) in a fresh status word, returned in *status.  The kernel then returns
 * normally: the context stays usable.  Synchronises `stream`. */
sat_status sat_diag_bounded_wait(uint32_t limit_us, uint32_t* status, void* stream);
/* Diagnostic of the initialisation's sign shortcut (the round kernel's threshold bits of
 * inputs outside every output's cone): at each of the 2^24 Box-Muller angles 2 pi k / 2^24,
 * compares the signs (-1, 0, +1) of the sine and cosine that sincospif returns (as the
 * normal draws compute them) with those read off k; *mismatches = the number of
 * disagreements (0 expected).  Synchronises `stream`. */
sat_status sat_diag_angle_signs(uint32_t* mismatches, void* stream);
/* Elements of one act / adj scratch array for a batch of B samples (enough for
 * either array under every call that takes them without a segment: max(n_cone,
 * adj rows) rows per tile). */
sat_status sat_plan_scratch_elems(const sat_plan* p, int64_t B, uint64_t* elems);
/* Exact sizes: act_elems (nullable) = elements of the act array of the fused steps
 * with recomputation segment `segment` (0 = every level stored: the layout of
 * sat_forward / sat_steps), adj_elems (nullable) = elements of the adj array (a ring
 * of max_span + 1 gate levels plus the input level, the same for every call).  A
 * segment > 0 builds and uploads that layout on first use (synchronous device
 * allocations and copies: make the first call before any stream capture). */
sat_status sat_plan_layout_elems(const sat_plan* p, int32_t segment, int64_t B, uint64_t* act_elems,
                                 uint64_t* adj_elems);
/* Which kernel runs the fused steps of this plan (sat_steps, sat_steps_aged,
 * sat_steps_recompute, sat_steps_noalloc and the rounds of sat_sample_plan).
 *   TILED: one CTA (or a 2-CTA cluster) per 128-sample tile, the activations and
 *     adjoints in the tile's act / adj scratch in device memory, rows staged through
 *     shared memory by TMA gathers.
 *   RESIDENT: one CTA per 32 samples, every activation, adjoint and the inputs' V, m, v
 *     in shared memory for all the launch's steps (device memory sees V, m, v read and
 *     written once, and the loss); for circuits whose state fits: 32 x (cone nodes x
 *     activation bytes + adjoint rows x 4 + cone inputs x 12) bytes <= 200 KiB.  The
 *     act / adj scratch is then left untouched.
 *   AUTO (the default): RESIDENT when the plan fits it with the call's act_dtype, else
 *     TILED.
 * Both kernels perform the same operations in the same order: V, m, v and the loss are
 * bit-identical.  SAT_STEP_KERNEL_RESIDENT is refused (SAT_ERR_ARG) for a plan that fits it
 * with no act_dtype; a step call whose act_dtype does not fit it returns SAT_ERR_CUDA.
 * Set it before, not during, calls that use the plan.  sat_plan_step_kernel reports the
 * kernel a step call with act_dtype would use (TILED or RESIDENT). */
typedef enum { SAT_STEP_KERNEL_AUTO = 0, SAT_STEP_KERNEL_TILED = 1, SAT_STEP_KERNEL_RESIDENT = 2 } sat_step_kernel;
sat_status sat_plan_set_step_kernel(sat_plan* p, int32_t kind);
sat_status sat_plan_step_kernel(const sat_plan* p, int32_t act_dtype, int32_t* kind);
void sat_plan_free(sat_plan* p);

/* ------------------------------------------- hot-path kernels (device) ---
 * All buffers are caller-owned device memory; B >= 0 samples. */

/* V[r][b] = scale * z_k, k = b mod 4: the Philox4x32-10 block (Salmon et al.,
 * SC'11) at counter (b / 4, r, round, 0) with key (seed low, seed high) gives
 * four standard normals z_0 .. z_3 as two Box-Muller pairs (cos, sin) of its
 * words (x, y) and (z, w), u1 = ((first >> 8) + 1) / 2^24, u2 = (second >> 8) /
 * 2^24.  Initial distribution: the paper does not state one; this is the
 * library's choice. */
sat_status sat_init_normal(const sat_plan* p, uint64_t seed, uint32_t round, float scale, float* V, int64_t ldv,
                           int64_t B, void* stream);

/* Eq. 5-7: act[i] = sigmoid(V[cone input i]), every cone gate by Table 1,
 * loss[b] = sum_j (Y_j - T_j)^2 accumulated in FP32 (loss nullable).  act holds
 * act_dtype elements; arithmetic is FP32. */
sat_status sat_forward(const sat_plan* p, sat_act_dtype act_dtype, const float* V, int64_t ldv, void* act,
                       float* loss, int64_t B, void* stream);

/* Eq. 8 (chain rule with the Table 1 derivatives): gV[r][b] = d(sum_b w_b
 * loss_b)/dV[r][b] with w = grad_loss (NULL = all ones), from the act written
 * by sat_forward.  adj: float32 scratch (sat_plan_layout_elems; its contents are
 * undefined afterwards).  Rows of gV outside the cone are not written (their
 * gradient is zero). */
sat_status sat_backward(const sat_plan* p, sat_act_dtype act_dtype, const float* V, int64_t ldv, const void* act,
                        float* adj, const float* grad_loss, float* gV, int64_t B, void* stream);

typedef struct sat_opt_params {
    int32_t optimizer;         /* sat_optimizer */
    float lr, beta1, beta2, eps;
} sat_opt_params;

/* One update of the cone rows of V at step t >= 1: GD (Eq. 9) V -= lr gV, or
 * Adam (PyTorch's formulation, no weight decay) on state m, v. */
sat_status sat_opt_update(const sat_plan* p, const sat_opt_params* o, float* V, float* m, float* v, const float* gV,
                          int64_t ldv, int32_t t, int64_t B, void* stream);

/* The fused hot loop: n_steps x (forward, loss, adjoint, update) at steps
 * t0 .. t0 + n_steps - 1, one kernel launch.  loss (nullable) receives the
 * per-sample loss of the last step's forward pass.  act and adj are scratch
 * (sat_plan_scratch_elems / sat_plan_layout_elems elements, 16-byte aligned):
 * their contents are undefined after the call (rows are dropped from L2 once
 * their last reader has run). */
sat_status sat_steps(const sat_plan* p, sat_act_dtype act_dtype, const sat_opt_params* o, float* V, float* m,
                     float* v, int64_t ldv, void* act, float* adj, float* loss, int32_t t0, int32_t n_steps,
                     int64_t B, void* stream);

/* sat_steps with per-sample Adam step counts, for early exit (below), where
 * samples restart at different times: the Adam step of sample b at in-launch
 * step s is age[b] + t0 + s (age: device int32 [B], read only; NULL = sat_steps).
 * GD ignores age. */
sat_status sat_steps_aged(const sat_plan* p, sat_act_dtype act_dtype, const sat_opt_params* o, float* V, float* m,
                          float* v, int64_t ldv, void* act, float* adj, float* loss, const int32_t* age, int32_t t0,
                          int32_t n_steps, int64_t B, void* stream);

/* sat_steps_aged with level-segment recomputation (segment > 0): the forward pass
 * keeps, of the gate levels, only the top max_span levels of every segment of
 * `segment` levels (the inputs of the next segment) and the levels holding outputs;
 * the backward pass evaluates each segment's other levels again (Eqs. 5-6, the same
 * arithmetic in the same order) before its adjoints.  Results are bit-identical to
 * sat_steps_aged; act needs sat_plan_layout_elems(p, segment, B) elements instead of
 * the full layout, for about (1 - max_span/segment) of a forward pass more work per step.
 * segment = 0 is sat_steps_aged, and so is a segment whose layout would not be smaller
 * than the full one (segment <= max_span, or segments so long that the two scratch
 * buffers outweigh the levels saved).  The paper stores every activation (autograd);
 * this is a memory schedule for circuits x batches beyond device memory. */
sat_status sat_steps_recompute(const sat_plan* p, sat_act_dtype act_dtype, const sat_opt_params* o, float* V,
                               float* m, float* v, int64_t ldv, void* act, float* adj, float* loss,
                               const int32_t* age, int32_t t0, int32_t n_steps, int64_t B, int32_t segment,
                               void* stream);

/* Early exit: verify every k steps, harvest the valid samples and give their
 * slots (and those of samples that have not converged after max_age steps) a
 * new start.  The paper stops "upon convergence" per sample (end of Section
 * III-A) without saying how a batch does it; this is the batched form.
 * sat_retire: restart bit b = valid bit b or age[b] + k >= max_age; age[b]
 * becomes 0 where restarting, else age[b] + k.  valid, restart: device uint32
 * [ceil(B/32)] (bit j of word w = sample 32w + j); age: device int32 [B]. */
sat_status sat_retire(const uint32_t* valid, int32_t* age, uint32_t* restart, int32_t k, int32_t max_age, int64_t B,
                      void* stream);
/* New starts for the samples whose restart bit is set: V[:, b] = src[:, b] when
 * src (device float [n_pi][lds]) is given, else init_scale * N(0,1) from the
 * Philox stream of round `round` (exactly what sat_init_normal draws for b);
 * m[:, b] = v[:, b] = 0.  Other samples are untouched. */
sat_status sat_restart(const sat_plan* p, const uint32_t* restart, uint64_t seed, uint32_t round, float init_scale,
                       const float* src, int64_t lds, float* V, float* m, float* v, int64_t ldv, int64_t B,
                       void* stream);

/* The same fused steps as sat_steps, for callers that cannot allocate device
 * memory when they run the optimiser (for example, a process whose device
 * budget belongs to another allocator, or a loop that must not wait for the
 * device synchronisation of cudaMalloc).  The paper has no counterpart: this is
 * a deployment variant.  The act/adj scratch comes from one fixed array of
 * SAT_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that loads the
 * library holds until the process exits; the call itself allocates nothing.
 * The arguments are those of sat_steps without act/adj, checked the same way
 * (SAT_ERR_ARG for a plan of another device than the current one, bad
 * optimiser parameters, NULL buffers).  A plan whose fused steps run on the
 * shared-memory resident kernel (sat_plan_step_kernel) needs no scratch and
 * is not limited by the array.  For the tiled kernel, a plan and batch whose
 * act/adj scratch exceeds the array (sat_plan_scratch_elems: the same rows,
 * each block rounded up to 256 bytes) are rejected with SAT_ERR_ARG before
 * any launch.  The first call on a device that needs the array looks up its
 * device address (cudaGetSymbolAddress) and keeps it for the process, so make
 * that first call before any stream capture, and do not use the library
 * across a cudaDeviceReset (which also frees every plan).  All calls share the
 * array: calls whose executions overlap on the GPU (other streams, other
 * threads) race and give undefined results.  Nothing in the array needs
 * clearing: every scratch row is written before it is read. */
#define SAT_NOALLOC_SCRATCH_BYTES (64u << 20)
sat_status sat_steps_noalloc(const sat_plan* p, sat_act_dtype act_dtype, const sat_opt_params* o, float* V, float* m,
                             float* v, int64_t ldv, float* loss, int32_t t0, int32_t n_steps, int64_t B,
                             void* stream);

/* Hard threshold (end of Section III-A): bit = [V > 0] (sigmoid(V) > 1/2; ties
 * give 0).  node_bits rows 0..n_pi-1 receive the bitsliced inputs; keys[b]
 * (key_words uint32 per sample, bit j of word k = input 32k + j) the packed
 * input vector used for deduplication. */
sat_status sat_threshold(const sat_plan* p, const float* V, int64_t ldv, uint32_t* node_bits, int64_t ldw,
                         uint32_t* keys, int64_t B, void* stream);

/* Boolean evaluation of every gate (constrained and unconstrained paths,
 * Fig. 1(b)) from the input rows of node_bits; rows n_pi..n_nodes-1 written. */
sat_status sat_hard_eval(const sat_plan* p, uint32_t* node_bits, int64_t ldw, int64_t B, void* stream);

/* Exact check against the ORIGINAL CNF: valid bit b = 1 iff the full
 * assignment of sample b satisfies every clause.  valid: [ceil(B/32)] words,
 * overwritten (padding bits 0). */
sat_status sat_cnf_check(const sat_plan* p, const uint32_t* node_bits, int64_t ldw, uint32_t* valid, int64_t B,
                         void* stream);

/* ------------------------------------ instance-compiled round (plain GD) ---
 * One sampling round of the paper's own setting (Section IV: plain gradient descent on V,
 * Eq. 9, for a few iterations) in ONE kernel launch (two when V is requested: the init
 * kernel writes every input's initial logit first), for small circuits.  The plan's
 * circuit is generated into the kernel's code (one thread per sample, every logit,
 * activation and adjoint in registers; indices as immediates) and compiled at run time
 * with NVRTC for sm_103a on first use.  It computes, with the same device functions in
 * the same order:
 *   sat_init_normal(seed, round, init_scale) ; sat_steps(FP32 activations, GD lr, n_steps) ;
 *   sat_threshold ; sat_hard_eval ; sat_cnf_check
 * so keys, valid and (when V != NULL) the final logits are bit-identical to those calls
 * run one after another.  Keys: [B][key_words] uint32 (bit j of word k = input 32k + j);
 * valid: [ceil(B/32)] words, overwritten (padding bits 0); V: nullable [n_pi][ldv],
 * ldv >= B, receives every input's final logit.  Nothing else is read or written.
 *
 * A plan has the kernel when its circuit is within the generator's limits: at most 256
 * primary inputs, cone inputs + cone nodes <= 224, at most 4,096 gates and 16,384
 * clause literals (sat_plan_round_info: available).  Errors: SAT_ERR_ARG for a plan
 * without it, NULL keys / valid, n_steps < 0, a non-finite lr or init_scale, or the
 * checks of every per-step call; SAT_ERR_CUDA when NVRTC or the module load fails (the
 * message holds the compiler log) or the launch fails.  The first call compiles (tens to
 * hundreds of ms, synchronous); make it before any stream capture.  Compiled programs are
 * cached per process by their text (the 32 most recently used): plans of the same circuit,
 * such as those sat_sample builds per call, compile once; sat_release_cached_memory drops
 * the cache (a plan keeps its own program loaded until it is freed).
 *
 * sat_sample_plan runs its rounds through this kernel when the plan has it, it compiled
 * without register spills, the plan's step kernel is AUTO, and the options ask for plain
 * GD on FP32 activations without a proposal, initial logits or early exit; its stats
 * then count the whole round as ms_steps. */
typedef struct sat_round_info {
    int32_t available;     /* 1: the plan's circuit is within the limits and has a round kernel */
    int32_t compiled;      /* 1: compiled and loaded (after a call with compile != 0 or a round) */
    int32_t registers;     /* registers per thread of the compiled kernel */
    int32_t spill_bytes;   /* local-memory bytes per thread (0: everything stays in registers) */
    int32_t min_blocks;    /* resident blocks of 128 threads per SM the kernel was compiled for: after
                              the first compilation, ptxas is asked for one block more (twice at most)
                              as long as that leaves no spills */
    double compile_ms;     /* NVRTC compilation(s) and module load */
} sat_round_info;
/* Host only (no device needed): compile == 0 writes the generated CUDA C++ program of the
 * circuit's round kernel; compile != 0 compiles it with NVRTC for sm_103a and writes the
 * compiler's log instead (with ptxas's register and spill report); SAT_ERR_CUDA when the
 * compilation fails, SAT_ERR_ARG for a circuit beyond the limits.  At most cap bytes are
 * written (NUL-terminated when they fit); *len = full length. */
sat_status sat_circuit_round_program(const sat_circuit* c, int32_t compile, char* buf, size_t cap, size_t* len);
/* compile != 0: compile and load now if not done yet (SAT_ERR_CUDA if that fails). */
sat_status sat_plan_round_info(const sat_plan* p, int32_t compile, sat_round_info* info);
sat_status sat_round_gd(const sat_plan* p, float lr, int32_t n_steps, uint64_t seed, uint32_t round,
                        float init_scale, float* V, int64_t ldv, uint32_t* keys, uint32_t* valid, int64_t B,
                        void* stream);

/* ----------------------------------------------------- deduplication ---
 * Device hash set of distinct solutions ("non-redundant", end of Section
 * III-A), keyed by the packed primary-input bits (the full assignment is a
 * function of them and contains them, so both are unique together).  Hash =
 * SplitMix64 finaliser fold (Steele, Lea, Flood 2014): h = 0x9E3779B97F4A7C15;
 * h = mix(h + w) over 64-bit key words w; h = mix(h ^ n_words).  Open
 * addressing with linear probing and full-key comparison; the probe count is
 * bounded, and a batch that would overflow max_keys is refused on the host
 * with SAT_ERR_TABLE_FULL before any kernel runs. */
sat_status sat_dedup_create(const sat_plan* p, uint64_t max_keys, int64_t max_batch, sat_dedup** out);
/* Inserts the valid rows of keys [B][key_words] (device).  hashes[b] (nullable,
 * device) = the key hash (0 for invalid rows); is_new[b] (nullable, device) =
 * 1 iff row b was inserted now.  Synchronises `stream` to check capacity. */
sat_status sat_dedup_insert(sat_dedup* d, const uint32_t* keys, const uint32_t* valid, int64_t B, uint64_t* hashes,
                            uint8_t* is_new, void* stream);
/* Number of stored keys (synchronises `stream`). */
sat_status sat_dedup_count(const sat_dedup* d, uint64_t* n, void* stream);
/* sat_dedup_insert without its two host synchronisations (the capacity check before the
 * launch and the status read after it), for loops that keep the device busy: the kernels
 * guard the pool on the device, and a batch that did not fit or hit the probe limit is
 * recorded in the set's status word (its keys are then incomplete).  sat_dedup_check
 * synchronises the stream and returns SAT_ERR_TABLE_FULL if any insert so far failed.
 * Inserts into one set share its scratch: issue them on one stream (or synchronise
 * between streams) so that they do not overlap. */
sat_status sat_dedup_insert_async(sat_dedup* d, const uint32_t* keys, const uint32_t* valid, int64_t B,
                                  void* stream);
sat_status sat_dedup_check(const sat_dedup* d, void* stream);
/* Copies stored keys [first, first+count) to host memory (synchronous). */
sat_status sat_dedup_copy_keys(const sat_dedup* d, uint64_t first, uint64_t count, uint32_t* host_keys, void* stream);
sat_status sat_dedup_clear(sat_dedup* d, void* stream);
void sat_dedup_free(sat_dedup* d);

/* ------------------------------------------------- proposal network ---
 * Learned proposal (not in the paper; a deployment option of this library):
 * an MLP maps Gaussian noise to initial logits V0.  Its layers run on the
 * tensor cores through this BF16 GEMM (tcgen05, FP32 accumulation in tensor
 * memory) with a fused epilogue:
 *   D[m][n] = sum_k A[m][k] B[n][k]  (A: [M][lda], B: [N][ldb], bf16, K-major,
 *                                     16-byte aligned, lda/ldb multiples of 8)
 *   x = alpha * epi(D + bias[n]),  epi: 0 identity, 1 GELU (erf form; D+bias
 *   is stored to pre[m][n] when pre != NULL), 2 multiply by GELU'(pre[m][n]).
 * x goes to any of out_f32 / out_bf16 ([M][ldo]) and out_t_bf16 / out_t_f32
 * (transposed, [N][ldt]); NULL outputs are skipped.  status (device uint32)
 * gets bit 3 if a bounded wait expired.  All pointers are device pointers. */
sat_status sat_gemm_bf16(int32_t M, int32_t N, int32_t K, const void* A, int64_t lda, const void* B, int64_t ldb,
                         const float* bias, int32_t epilogue, float* pre, int64_t ldpre, float alpha, float* out_f32,
                         void* out_bf16, int64_t ldo, void* out_t_bf16, float* out_t_f32, int64_t ldt,
                         uint32_t* status, void* stream);

/* The proposal network: z (n_in) -> GELU(W1 z + b1) -> GELU(W2 . + b2) ->
 * W3 . + b3 = logits of the n_out primary inputs.  FP32 master weights with
 * BF16 copies; BF16 activations; FP32 accumulation; PyTorch's nn.Linear
 * initialisation from `seed`.  max_rows bounds every batch the object handles
 * (inference rows, or training targets x candidates).  Training is implicit
 * maximum likelihood (IMLE): for each training solution draw K noise vectors,
 * keep the one whose logits have the least summed binary cross-entropy to the
 * solution's input bits, and take an Adam step on the mean BCE at the kept
 * vectors.  Solutions are passed as dedup keys (device uint32 [S][key_words],
 * bit i = primary input i).  Parameter vector order: W1 [h][n_in], b1, W2
 * [h][h], b2, W3 [n_out][h], b3. */
sat_status sat_mlp_create(uint32_t n_in, uint32_t n_hidden, uint32_t n_out, int64_t max_rows, uint64_t seed,
                          sat_mlp** out);
sat_status sat_mlp_num_params(const sat_mlp* m, uint64_t* n);
sat_status sat_mlp_get_params(const sat_mlp* m, float* host);            /* host [n_params] */
sat_status sat_mlp_set_params(sat_mlp* m, const float* host);            /* also resets Adam state */
/* z [rows][n_in] bf16 ~ N(0,1): the Philox4x32-10 block at counter (row, c, round, 1) gives
 * z[row][4c .. 4c+3] as two Box-Muller pairs (cos, sin) of its words (x, y) and (z, w). */
sat_status sat_mlp_draw_noise(sat_mlp* m, uint64_t seed, uint32_t round, void* z, int64_t rows, void* stream);
/* V[i][b] = tau * logit_i(z_b) for rows b < rows (V: float [n_out][ldv], the sampler's layout). */
sat_status sat_mlp_forward(sat_mlp* m, const void* z, int64_t rows, float tau, float* V, int64_t ldv, void* stream);
/* Draw noise and write tau * logits into V: the proposal's initial logits for a round. */
sat_status sat_mlp_propose(sat_mlp* m, uint64_t seed, uint32_t round, float tau, float* V, int64_t ldv, int64_t B,
                           void* stream);
/* IMLE selection: candidate k of target s is row s*K+k of zc; dist[s*K+k] =
 * summed BCE (device, nullable), choice[s] = first argmin (device, nullable). */
sat_status sat_mlp_imle_select(sat_mlp* m, const void* zc, const uint32_t* keys, int32_t key_words, int64_t S,
                               int32_t K, float* dist, int32_t* choice, void* stream);
/* Mean BCE and its gradient at noise rows z [S][n_in] (device bf16); loss_host
 * and grad_host ([n_params]) are host pointers (nullable).  Synchronises. */
sat_status sat_mlp_loss_grad(sat_mlp* m, const void* z, const uint32_t* keys, int32_t key_words, int64_t S,
                             float* loss_host, float* grad_host, void* stream);
/* One Adam step of the master weights with a given gradient grad (device float
 * [n_params], the parameter order above): step count t = previous + 1, then
 *   m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
 *   theta <- theta - lr / (1 - b1^t) * m / (sqrt(v) / sqrt(1 - b2^t) + eps)
 * with b1 = 0.9f, b2 = 0.999f, eps = 1e-8f (PyTorch's Adam, no weight decay; the
 * betas are these FP32 values in every term, bias corrections included); the
 * BF16 copies of the weights are refreshed.  The paper has no learned part; the
 * optimiser is the one the proposal's configuration names. */
sat_status sat_mlp_apply_grad(sat_mlp* m, const float* grad, float lr, void* stream);
/* One IMLE step with K candidates per target: sat_mlp_imle_select on fresh noise,
 * sat_mlp_loss_grad at the chosen rows, then sat_mlp_apply_grad with that gradient. */
sat_status sat_mlp_train_step(sat_mlp* m, const uint32_t* keys, int32_t key_words, int64_t S, int32_t K, float lr,
                              uint64_t seed, uint32_t round, float* loss_host, void* stream);
/* Train the proposal on distinct solutions: sols holds n full assignments in the
 * sat_solutions_copy format (host uint64 words, ceil(n_vars/64) per solution) of the
 * circuit the plan p was made from; their primary-input bits (in p's input order, the
 * network's outputs) are the targets.  `steps` IMLE steps (sat_mlp_train_step) of S targets
 * drawn uniformly with replacement (SplitMix64 of seed) and K candidates each, learning rate
 * lr; loss_host (nullable) receives the last step's mean loss.  S*K must be <= max_rows.
 * Each step's S targets are gathered on the host and copied in; synchronises the stream at the end. */
sat_status sat_mlp_train(sat_mlp* m, const sat_plan* p, const uint64_t* sols, uint64_t n, int32_t steps, int64_t S,
                         int32_t K, float lr, uint64_t seed, float* loss_host, void* stream);
/* Status word of the network's kernels (bit 3: a bounded GEMM wait expired). */
sat_status sat_mlp_status(const sat_mlp* m, uint32_t* status);
void sat_mlp_free(sat_mlp* m);

/* -------------------------------------------------------- end to end ---
 * The sampling problem of Section II-A: draw many distinct assignments that
 * satisfy every clause of a CNF.  The method of Section III-A learns a batch
 * of input vectors on the relaxed circuit (Eqs. 5-9), thresholds them, and
 * keeps only the satisfiable, non-redundant rows (the end of Section III-A);
 * Section IV measures it as unique valid solutions per second.  Here that is
 * rounds of: init (or caller logits, or the proposal network) -> `steps`
 * fused steps -> threshold -> Boolean pass -> exact check against the
 * original clauses -> dedup, until n_wanted distinct solutions or max_rounds.
 * Round r draws its initial logits (or the proposal's noise) with round
 * counter first_round + r.  Returns SAT_PARTIAL (with what was found) when the
 * budget ends first.  The stats' device times give the throughput of Section
 * IV (distinct solutions over time; the host transformation is timed apart by
 * sat_circuit_build, as the paper reports it separately in Section IV-C). */
typedef struct sat_sample_opts {
    int64_t batch;
    int32_t steps;
    int32_t max_rounds;
    sat_opt_params opt;
    uint64_t seed;
    uint32_t first_round;
    float init_scale;
    int32_t act_dtype;          /* sat_act_dtype */
    int32_t steps_per_launch;   /* 0 = all steps in one launch */
    const float* init_logits;   /* nullable device [n_pi][init_ld]: used instead of init for round 0 */
    int64_t init_ld;
    void* stream;
    sat_mlp* proposal;          /* nullable: initial logits from the proposal network (max_rows >= batch) */
    float proposal_tau;         /* scale of the proposal's logits */
    int32_t check_every;        /* > 0: early exit, verify every check_every steps (see sat_retire);
                                   the budget stays max_rounds x steps descent steps of the batch */
    int32_t max_age;            /* early exit: restart samples unsolved after max_age steps (0 = steps) */
    int32_t recompute_segment;  /* > 0: level-segment recomputation (sat_steps_recompute); 0 = store all */
    int32_t step_kernel;        /* sat_sample: sat_step_kernel of the plan it builds (sat_sample_plan uses
                                   the plan's own setting) */
} sat_sample_opts;

typedef struct sat_sample_stats {
    uint32_t rounds;                   /* rounds, or verification epochs under early exit */
    uint64_t samples, valid, unique;   /* samples started, valid harvests (with repeats), distinct */
    double ms_init, ms_steps, ms_verify, ms_dedup, ms_total;   /* device time per phase (CUDA events) */
    double ms_upload, ms_download;                              /* sat_sample only */
} sat_sample_stats;

/* Device memory.  The workspace of sat_sample / sat_sample_plan (and the buffers that
 * order sat_sample's solutions), and the arrays of plans and dedup sets, come from the
 * library's own stream-ordered pool on the current device (plans and dedup sets are
 * allocated and freed in order on the legacy default stream), which keeps the memory it
 * has reserved when those buffers are freed, so a repeated call maps no new device memory
 * and freeing does not wait for the device.  sat_cached_memory reports the
 * pool's reserved and in-use bytes; sat_release_cached_memory returns the reserve that no
 * allocation (or queued work) still uses to the device, and frees the host buffers kept
 * between calls: the pinned buffer that solutions are downloaded through and the key
 * buffers of up to two freed solution sets (1 MiB-256 MiB each), which the next
 * sat_sample reuses; it also drops the cache of compiled round programs (sat_round_gd).
 * Proposal networks are allocated separately (cudaMalloc). */
sat_status sat_cached_memory(uint64_t* reserved_bytes, uint64_t* used_bytes);
sat_status sat_release_cached_memory(void);

/* Defaults: batch 1,024, 200 steps, 1 round, Adam lr 0.1 (beta 0.9/0.999, eps 1e-8),
 * seed 0, init_scale 1, FP32 activations, no early exit, no recomputation. */
void sat_sample_opts_default(sat_sample_opts* o);
/* The whole sampler from host objects (Section III-A, end to end): builds a plan
 * of circuit c for cnf (the clauses that are checked are cnf's own), samples
 * until n_wanted distinct solutions or the round budget, and returns them in
 * *out (owned by the caller, freed with sat_solutions_free).  SAT_OK when
 * n_wanted were found, SAT_PARTIAL with fewer; SAT_ERR_ARG on bad options
 * (batch < 1, steps < 0, max_rounds < 1, bad optimiser), SAT_ERR_OOM when the
 * workspace does not fit on the device, SAT_ERR_CUDA on a device error (out is
 * then NULL).  stats (nullable) gets counts and per-phase device times.  Runs on
 * o->stream of the current device and synchronises it before returning. */
sat_status sat_sample(const sat_circuit* c, const sat_cnf* cnf, const sat_sample_opts* o, uint64_t n_wanted,
                      sat_solutions** out, sat_sample_stats* stats);
/* The same rounds on an existing plan, adding the distinct solutions to an existing
 * dedup set d (device-resident: nothing is copied to the host; read d with
 * sat_dedup_count / sat_dedup_copy_keys).  n_wanted counts d's total.  Errors as
 * sat_sample, plus SAT_ERR_TABLE_FULL when d cannot take a round's distinct keys. */
sat_status sat_sample_plan(const sat_plan* p, sat_dedup* d, const sat_sample_opts* o, uint64_t n_wanted,
                           sat_sample_stats* stats);

/* The kept rows of Section III-A's last step: satisfiable (every original clause
 * has a true literal) and non-redundant (pairwise distinct full assignments).
 * sat_solutions_count: their number (0 for NULL); sat_solutions_nvars: variables
 * of each assignment (the CNF's). */
uint64_t sat_solutions_count(const sat_solutions* s);
uint32_t sat_solutions_nvars(const sat_solutions* s);
/* Full assignments of solutions [first, first+count) in canonical ascending
 * order (of the packed primary-input bits, the dedup key): ceil(n_vars/64)
 * uint64 words each into host words_out, bit j of word k = variable 64k+j+1.
 * SAT_ERR_ARG when the range exceeds the count or an argument is NULL. */
sat_status sat_solutions_copy(const sat_solutions* s, uint64_t first, uint64_t count, uint64_t* words_out);
/* Frees a solution set (NULL is accepted). */
void sat_solutions_free(sat_solutions* s);

#ifdef __cplusplus
}
#endif
#endif /* SATSAMPLER_H */
