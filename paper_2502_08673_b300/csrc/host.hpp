// Internal host-side data structures of the sampler library (not part of the C ABI).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace sat {

// ---------------------------------------------------------------- CNF ----
struct Cnf {
    uint32_t n_vars = 0;
    std::vector<int64_t> off;   // clause c holds lits[off[c] .. off[c+1])
    std::vector<int32_t> lits;  // signed DIMACS literals
    size_t n_clauses() const { return off.empty() ? 0 : off.size() - 1; }
};

// Parses DIMACS text; on failure returns false and sets err.
bool parse_dimacs(const char* buf, size_t len, Cnf& out, std::string& err);

// ------------------------------------------------------- truth tables ----
// Truth table over at most 8 support variables: bit x of the table is the
// function's value on the assignment whose bit i is support variable i.
struct TT {
    uint64_t w[4] = {0, 0, 0, 0};
    static TT full(int k);
    static TT var(int i, int k);
    TT operator&(const TT& o) const { TT r; for (int i = 0; i < 4; i++) r.w[i] = w[i] & o.w[i]; return r; }
    TT operator|(const TT& o) const { TT r; for (int i = 0; i < 4; i++) r.w[i] = w[i] | o.w[i]; return r; }
    TT andnot_of(const TT& fullmask) const { TT r; for (int i = 0; i < 4; i++) r.w[i] = fullmask.w[i] & ~w[i]; return r; }
    bool operator==(const TT& o) const { return w[0] == o.w[0] && w[1] == o.w[1] && w[2] == o.w[2] && w[3] == o.w[3]; }
    bool operator!=(const TT& o) const { return !(*this == o); }
    bool bit(unsigned x) const { return (w[x >> 6] >> (x & 63)) & 1; }
    void set(unsigned x) { w[x >> 6] |= 1ull << (x & 63); }
    int popcount() const;
};

// ------------------------------------------------------------ circuit ----
enum DefKind : uint8_t { K_LIT = 0, K_AND = 1, K_OR = 2, K_XOR = 3, K_SOP = 4 };

struct Def {
    uint32_t var = 0;
    DefKind kind = K_LIT;
    bool out_neg = false;
    std::vector<int32_t> lits;                 // LIT/AND/OR/XOR operands (signed var ids)
    std::vector<std::vector<int32_t>> terms;   // SOP product terms
    std::vector<uint32_t> support;             // ascending var ids the function depends on
    TT table;                                  // truth table over support
};

struct Circuit {
    uint32_t n_vars = 0;
    std::vector<uint32_t> pis;                    // ascending var ids
    std::vector<Def> defs;                        // acceptance order (topological)
    std::vector<std::vector<int32_t>> outputs;    // OR outputs constrained to 1
    uint32_t n_const = 0;                         // constant acceptances
    double wall_ms = 0.0;
};

struct TransformOpts {
    uint32_t max_support = 8;
    uint32_t max_window = 16;
    bool direct = false;   // no factorization: clauses as OR outputs, all variables inputs
    bool reorder = false;  // sort clauses by (largest variable, position) first
};

// Algorithm 1 with the fallback for under-specified clauses.
bool transform(const Cnf& cnf, const TransformOpts& o, Circuit& out, std::string& err);

// Canonical text form (used to compare against an independent implementation).
std::string circuit_dump(const Circuit& c);

// ---------------------------------------------------------- schedule ----
// 2-input gate encoding (one byte): op in bits 0-1 (0 AND, 1 OR, 2 XOR),
// input-0 negation in bit 2, input-1 negation in bit 3.
enum GateOp : uint8_t { G_AND = 0, G_OR = 1, G_XOR = 2 };

struct Plan {
    // Full node space: primary inputs 0..n_pi-1 (ascending var id), then every
    // lowered 2-input gate in topological (level, creation) order.
    uint32_t n_vars = 0, n_pi = 0;
    uint64_t n_nodes = 0;
    std::vector<uint32_t> pi_var;                 // node -> DIMACS var, for PIs
    std::vector<int32_t> in0, in1;                // per gate (index = node - n_pi)
    std::vector<uint8_t> gop;                     // per gate
    std::vector<int32_t> level_off;               // full levels: gates of level l are nodes level_off[l]..level_off[l+1]
    std::vector<int32_t> var_node;                // DIMACS var -> node (index 0 unused)
    std::vector<uint8_t> var_neg;                 // DIMACS var -> literal negation
    // Outputs in order: Y_j = A[out_node[j]] compared with target[j] (0 or 1).
    std::vector<int32_t> out_node;                // full node ids
    std::vector<float> out_target;

    // Cone schedule (the part gradient descent touches), its own dense index space:
    // cone PIs 0..n_cone_pi-1 (ascending var id), then cone gates by level.
    uint32_t n_cone_pi = 0;
    uint64_t n_cone = 0;
    std::vector<int32_t> cone_pi_row;             // cone PI -> row of V (= full PI node id)
    std::vector<int32_t> c_in0, c_in1;            // per cone gate, cone indices
    std::vector<uint8_t> c_gop;
    std::vector<int32_t> c_level_off;             // level l (>= 1) gates are cone nodes c_level_off[l]..c_level_off[l+1]; level 0 = PIs
    std::vector<int32_t> c_out_node;              // outputs in cone index space
    // Fan-out CSR over cone nodes for the gather form of the adjoint.  Each
    // edge holds the consuming gate and the sibling input, with the partial
    // d g / d A_self = c0 + c1 * A_sibling (small integer coefficients).  An
    // edge with consumer -1 is an output seed 2 (A_self - target): sibling =
    // the node itself, c0 = -2 target, c1 = 2.
    std::vector<int64_t> fo_off;
    std::vector<int32_t> fo_g, fo_sib;
    std::vector<int8_t> fo_c0, fo_c1;
    uint32_t max_span = 0;                        // max level distance of a cone edge

    // CNF in node space for the bitsliced clause check.
    std::vector<int64_t> cl_off;
    std::vector<int32_t> cl_node;                 // literal -> full node
    std::vector<uint8_t> cl_neg;                  // literal negation relative to the node
    uint64_t ops_cnf = 0, ops_circuit = 0;
};

bool build_plan(const Circuit& c, const Cnf& cnf, Plan& out, std::string& err);

}  // namespace sat

// Shared by the C entry points defined outside capi.cpp.
#include "../../include/satsampler.h"
namespace sat {
struct DevPlan;
// Records msg as the calling thread's last error and returns s.
sat_status report_error(sat_status s, const std::string& msg);
// The device-side view of a plan.
const DevPlan* plan_device(const sat_plan* p);
// The checks every per-step entry point makes first: p not NULL, 0 <= B < 2^31, ldv >= B
// (ldv < 0: no V argument), and p's device is the current device (SAT_ERR_ARG otherwise).
sat_status check_plan_call(const sat_plan* p, int64_t B, int64_t ldv);
// Optimiser parameters the kernels accept (Adam with beta1, beta2 in [0, 1), or GD).
bool opt_params_ok(const sat_opt_params* o);
// The kernels' copy of checked optimiser parameters.
struct OptParams;
OptParams opt_params_of(const sat_opt_params* o);
}  // namespace sat
