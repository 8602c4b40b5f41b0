// Lowering of a transformed circuit to levelled 2-input gates, and the device
// schedule built from it.
//
// Relaxation (Table 1, Section III-A): every k-input AND/OR/XOR is evaluated
// as a left fold of 2-input gates over its operands; a sum of products is an
// OR fold of AND folds (the form of Fig. 1(c)).  The fold reproduces the
// k-input product formulas of Table 1's gates exactly in real arithmetic.
// Aliases (buffers, inverters) become literals of their source node.  Each
// OR output (a constraint clause) becomes one output node with its target.
//
// The "cone" is the fan-in cone of the outputs: the only nodes whose values
// reach the loss, so the only ones the gradient loop evaluates (constrained
// paths of Fig. 1(b)); the rest is evaluated in the Boolean pass only.
#include <algorithm>
#include <numeric>

#include "host.hpp"

namespace sat {

namespace {

struct Lit {
    int32_t node;
    uint8_t neg;
};

struct Lowering {
    uint32_t n_pi = 0;
    std::vector<int32_t> in0, in1;
    std::vector<uint8_t> op, n0, n1;
    Lit mk(uint8_t o, Lit a, Lit b) {
        in0.push_back(a.node);
        in1.push_back(b.node);
        op.push_back(o);
        n0.push_back(a.neg);
        n1.push_back(b.neg);
        return Lit{(int32_t)(n_pi + in0.size() - 1), 0};
    }
    Lit fold(uint8_t o, const std::vector<Lit>& ls) {
        Lit acc = ls[0];
        for (size_t i = 1; i < ls.size(); i++) acc = mk(o, acc, ls[i]);
        return acc;
    }
};

// Partial of gate output w.r.t. its input `self` as c0 + c1 * A_sibling.
void partial_coeffs(uint8_t op, uint8_t n_self, uint8_t n_sib, int8_t& c0, int8_t& c1) {
    int s = n_self ? -1 : 1;        // d q_self / d A_self
    int t = 1 - 2 * (int)n_sib;     // q_sib = n_sib + t * A_sib
    switch (op) {
    case G_AND:  // d/dq_self (q_self q_sib) = q_sib
        c0 = (int8_t)(s * n_sib);
        c1 = (int8_t)(s * t);
        break;
    case G_OR:   // 1 - q_sib
        c0 = (int8_t)(s * (1 - n_sib));
        c1 = (int8_t)(-s * t);
        break;
    default:     // XOR: 1 - 2 q_sib
        c0 = (int8_t)(s * (1 - 2 * n_sib));
        c1 = (int8_t)(-2 * s * t);
        break;
    }
}

}  // namespace

bool build_plan(const Circuit& c, const Cnf& cnf, Plan& P, std::string& err) {
    P = Plan();
    P.n_vars = c.n_vars;
    P.n_pi = (uint32_t)c.pis.size();
    Lowering low;
    low.n_pi = P.n_pi;
    std::vector<Lit> var_lit(c.n_vars + 1, Lit{-1, 0});
    for (uint32_t i = 0; i < P.n_pi; i++) var_lit[c.pis[i]] = Lit{(int32_t)i, 0};
    auto lit = [&](int32_t l) -> Lit {
        Lit r = var_lit[std::abs(l)];
        if (r.node < 0) return r;
        if (l < 0) r.neg ^= 1;
        return r;
    };
    auto lits = [&](const std::vector<int32_t>& ls, std::vector<Lit>& out) {
        out.clear();
        for (int32_t l : ls) {
            Lit r = lit(l);
            if (r.node < 0) return false;
            out.push_back(r);
        }
        return true;
    };
    std::vector<Lit> tmp;
    for (const Def& d : c.defs) {
        Lit r;
        if (d.kind == K_SOP) {
            std::vector<Lit> terms;
            for (const auto& t : d.terms) {
                if (!lits(t, tmp)) { err = "definition uses an undefined variable"; return false; }
                terms.push_back(tmp.size() == 1 ? tmp[0] : low.fold(G_AND, tmp));
            }
            r = terms.size() == 1 ? terms[0] : low.fold(G_OR, terms);
        } else {
            if (!lits(d.lits, tmp)) { err = "definition uses an undefined variable"; return false; }
            if (d.kind == K_LIT) r = tmp[0];
            else r = low.fold(d.kind == K_AND ? G_AND : d.kind == K_OR ? G_OR : G_XOR, tmp);
        }
        if (d.out_neg) r.neg ^= 1;
        var_lit[d.var] = r;
    }
    std::vector<Lit> outs;
    for (const auto& o : c.outputs) {
        if (!lits(o, tmp)) { err = "output uses an undefined variable"; return false; }
        outs.push_back(tmp.size() == 1 ? tmp[0] : low.fold(G_OR, tmp));
    }
    for (uint32_t v = 1; v <= c.n_vars; v++)
        if (var_lit[v].node < 0) { err = "variable left without a node"; return false; }

    // Levels and the full schedule (gates sorted by level, then creation order).
    const size_t G = low.in0.size();
    P.n_nodes = P.n_pi + G;
    std::vector<int32_t> lev(P.n_nodes, 0);
    int32_t L = 0;
    for (size_t g = 0; g < G; g++) {
        lev[P.n_pi + g] = 1 + std::max(lev[low.in0[g]], lev[low.in1[g]]);
        L = std::max(L, lev[P.n_pi + g]);
    }
    std::vector<int32_t> order(G);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return lev[P.n_pi + a] < lev[P.n_pi + b]; });
    std::vector<int32_t> newid(P.n_nodes);
    for (uint32_t i = 0; i < P.n_pi; i++) newid[i] = (int32_t)i;
    for (size_t r = 0; r < G; r++) newid[P.n_pi + order[r]] = (int32_t)(P.n_pi + r);
    P.in0.resize(G); P.in1.resize(G); P.gop.resize(G);
    std::vector<int32_t> flev(P.n_nodes, 0);
    for (size_t r = 0; r < G; r++) {
        int32_t g = order[r];
        P.in0[r] = newid[low.in0[g]];
        P.in1[r] = newid[low.in1[g]];
        P.gop[r] = (uint8_t)(low.op[g] | (low.n0[g] << 2) | (low.n1[g] << 3));
        flev[P.n_pi + r] = lev[P.n_pi + g];
    }
    P.level_off.assign(L + 2, 0);
    P.level_off[0] = 0;
    {
        size_t r = 0;
        for (int32_t l = 1; l <= L; l++) {
            P.level_off[l] = (int32_t)(P.n_pi + r);
            while (r < G && flev[P.n_pi + r] == l) r++;
        }
        P.level_off[L + 1] = (int32_t)(P.n_pi + r);
        P.level_off[0] = 0;
    }
    P.pi_var = c.pis;
    P.var_node.assign(c.n_vars + 1, 0);
    P.var_neg.assign(c.n_vars + 1, 0);
    for (uint32_t v = 1; v <= c.n_vars; v++) {
        P.var_node[v] = newid[var_lit[v].node];
        P.var_neg[v] = var_lit[v].neg;
    }
    for (const Lit& o : outs) {
        P.out_node.push_back(newid[o.node]);
        P.out_target.push_back(o.neg ? 0.0f : 1.0f);
    }

    // Cone of the outputs.
    std::vector<uint8_t> in_cone(P.n_nodes, 0);
    for (int32_t n : P.out_node) in_cone[n] = 1;
    for (int64_t r = (int64_t)G - 1; r >= 0; r--) {
        if (!in_cone[P.n_pi + r]) continue;
        in_cone[P.in0[r]] = 1;
        in_cone[P.in1[r]] = 1;
    }
    std::vector<int32_t> cidx(P.n_nodes, -1);
    for (uint32_t i = 0; i < P.n_pi; i++)
        if (in_cone[i]) {
            cidx[i] = (int32_t)P.cone_pi_row.size();
            P.cone_pi_row.push_back((int32_t)i);
        }
    P.n_cone_pi = (uint32_t)P.cone_pi_row.size();
    int64_t nc = P.n_cone_pi;
    int32_t CL = 0;
    P.c_level_off.assign(1, 0);
    std::vector<int32_t> clev;
    clev.assign(P.n_cone_pi, 0);
    for (size_t r = 0; r < G; r++) {
        uint64_t n = P.n_pi + r;
        if (!in_cone[n]) continue;
        cidx[n] = (int32_t)nc++;
        clev.push_back(flev[n]);
        CL = std::max(CL, flev[n]);
    }
    P.n_cone = (uint64_t)nc;
    P.c_in0.reserve(nc - P.n_cone_pi);
    for (size_t r = 0; r < G; r++) {
        uint64_t n = P.n_pi + r;
        if (!in_cone[n]) continue;
        P.c_in0.push_back(cidx[P.in0[r]]);
        P.c_in1.push_back(cidx[P.in1[r]]);
        P.c_gop.push_back(P.gop[r]);
    }
    // cone levels: level 0 = PIs [0, n_cone_pi); level l >= 1 from c_level_off[l]
    P.c_level_off.assign(CL + 2, 0);
    {
        int64_t i = P.n_cone_pi;
        for (int32_t l = 1; l <= CL; l++) {
            P.c_level_off[l] = (int32_t)i;
            while (i < nc && clev[i] == l) i++;
        }
        P.c_level_off[CL + 1] = (int32_t)nc;
        P.c_level_off[0] = 0;
    }
    for (int32_t n : P.out_node) P.c_out_node.push_back(cidx[n]);

    // Fan-out CSR (deterministic order: output seeds, then consumers by index, slot 0 first).
    // Every cone node has at least one edge (it is an output or feeds a cone gate); a node
    // without one would get a zero edge, so that each node's adjoint is stored at its last edge.
    std::vector<int64_t> deg(nc + 1, 0);
    for (int32_t n : P.c_out_node) deg[n]++;
    for (size_t g = 0; g < P.c_in0.size(); g++) {
        deg[P.c_in0[g]]++;
        deg[P.c_in1[g]]++;
    }
    std::vector<int64_t> zero_edge;
    for (int64_t i = 0; i < nc; i++)
        if (deg[i] == 0) {
            deg[i] = 1;
            zero_edge.push_back(i);
        }
    P.fo_off.assign(nc + 1, 0);
    for (int64_t i = 0; i < nc; i++) P.fo_off[i + 1] = P.fo_off[i] + deg[i];
    int64_t E = P.fo_off[nc];
    P.fo_g.assign(E, 0); P.fo_sib.assign(E, 0); P.fo_c0.assign(E, 0); P.fo_c1.assign(E, 0);
    std::vector<int64_t> fill(P.fo_off.begin(), P.fo_off.end() - 1);
    for (size_t j = 0; j < P.c_out_node.size(); j++) {
        // output seed 2 (A_u - T) = c0 + c1 * A_u with the node itself as "sibling"
        int64_t e = fill[P.c_out_node[j]]++;
        P.fo_g[e] = -1;
        P.fo_sib[e] = P.c_out_node[j];
        P.fo_c0[e] = (int8_t)(-2 * (int)P.out_target[j]);
        P.fo_c1[e] = 2;
    }
    uint32_t span = 0;
    for (size_t g = 0; g < P.c_in0.size(); g++) {
        int32_t gn = (int32_t)(P.n_cone_pi + g);
        uint8_t f = P.c_gop[g], op = f & 3, n0 = (f >> 2) & 1, n1 = (f >> 3) & 1;
        int64_t e0 = fill[P.c_in0[g]]++;
        P.fo_g[e0] = gn;
        P.fo_sib[e0] = P.c_in1[g];
        partial_coeffs(op, n0, n1, P.fo_c0[e0], P.fo_c1[e0]);
        int64_t e1 = fill[P.c_in1[g]]++;
        P.fo_g[e1] = gn;
        P.fo_sib[e1] = P.c_in0[g];
        partial_coeffs(op, n1, n0, P.fo_c0[e1], P.fo_c1[e1]);
        span = std::max<uint32_t>(span, (uint32_t)(clev[gn] - clev[P.c_in0[g]]));
        span = std::max<uint32_t>(span, (uint32_t)(clev[gn] - clev[P.c_in1[g]]));
    }
    P.max_span = span;
    for (int64_t i : zero_edge) {  // contribution 0 * (0 + 0 * A_i)
        int64_t e = fill[i]++;
        P.fo_g[e] = -1;
        P.fo_sib[e] = (int32_t)i;
        P.fo_c0[e] = 0;
        P.fo_c1[e] = 0;
    }

    // Original clauses in node space.
    P.cl_off.assign(cnf.n_clauses() + 1, 0);
    P.cl_node.resize(cnf.lits.size());
    P.cl_neg.resize(cnf.lits.size());
    for (size_t ci = 0; ci < cnf.n_clauses(); ci++) {
        P.cl_off[ci + 1] = cnf.off[ci + 1];
        for (int64_t i = cnf.off[ci]; i < cnf.off[ci + 1]; i++) {
            int32_t l = cnf.lits[i];
            uint32_t v = (uint32_t)std::abs(l);
            P.cl_node[i] = P.var_node[v];
            P.cl_neg[i] = (uint8_t)(P.var_neg[v] ^ (l < 0 ? 1 : 0));
        }
    }
    for (size_t ci = 0; ci < cnf.n_clauses(); ci++) P.ops_cnf += (uint64_t)(cnf.off[ci + 1] - cnf.off[ci] - 1);
    P.ops_cnf += cnf.n_clauses() ? cnf.n_clauses() - 1 : 0;
    P.ops_circuit = G + (outs.empty() ? 0 : outs.size() - 1);
    return true;
}

}  // namespace sat
