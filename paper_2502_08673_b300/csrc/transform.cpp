// Native transformation of a CNF into a multi-level, multi-output circuit:
// Algorithm 1 of Section III-A and the fallback for under-specified clauses
// that follows it.  The readings taken where the paper is silent:
//  * window candidates v are tried in descending variable id (every gate group
//    of Fig. 1 defines its largest variable);
//  * v = f is accepted when f, the conjunction of the clauses holding -v with
//    -v removed, is the complement of the expression found from the clauses
//    holding v; window clauses without v become constraint outputs;
//  * a constant f makes v a primary output (a unit constraint);
//  * the other variables of the defining clauses that are not intermediate
//    become primary inputs, as in Algorithm 1;
//  * with no definition, the window is emitted as OR outputs constrained to 1
//    when none of its variables occurs later, and is kept within max_window
//    clauses / max_support variables by emitting its oldest clause;
//  * optionally (reorder), clauses are first sorted by (largest variable,
//    longer first, position), which makes each defined variable's clauses
//    adjacent, ahead of unit clauses on it, when a file interleaves them;
//  * accepted functions are simplified to aliases, AND/OR/XOR of literals, or
//    a sum of products over a minimum prime cover (fewest terms, then fewest
//    literals, then first in (literal count, care mask, value) order; with more
//    than 20 primes, all of them).
#include <algorithm>
#include <chrono>
#include <set>
#include <tuple>
#include <sstream>
#include <unordered_set>

#include "host.hpp"

namespace sat {

TT TT::full(int k) {
    TT t;
    unsigned n = 1u << k;
    for (unsigned x = 0; x < n; x++) t.set(x);
    return t;
}

TT TT::var(int i, int k) {
    TT t;
    unsigned n = 1u << k;
    for (unsigned x = 0; x < n; x++)
        if ((x >> i) & 1) t.set(x);
    return t;
}

int TT::popcount() const {
    return __builtin_popcountll(w[0]) + __builtin_popcountll(w[1]) + __builtin_popcountll(w[2]) +
           __builtin_popcountll(w[3]);
}

namespace {

using Clause = std::vector<int32_t>;

int pos_of(const std::vector<uint32_t>& support, uint32_t v) {
    return (int)(std::lower_bound(support.begin(), support.end(), v) - support.begin());
}

// OR of the clause's literals except `skip`, as a table over `support`.
TT clause_table(const Clause& c, int32_t skip, const std::vector<uint32_t>& support) {
    int k = (int)support.size();
    TT full = TT::full(k), t;
    for (int32_t l : c) {
        if (l == skip) continue;
        TT m = TT::var(pos_of(support, (uint32_t)std::abs(l)), k);
        t = t | (l > 0 ? m : m.andnot_of(full));
    }
    return t;
}

// Conjunction, over clauses holding -lit, of the clause without -lit.
TT find_expression(int32_t lit, const std::vector<const Clause*>& cls, const std::vector<uint32_t>& support) {
    TT f = TT::full((int)support.size());
    for (const Clause* c : cls)
        if (std::find(c->begin(), c->end(), -lit) != c->end()) f = f & clause_table(*c, -lit, support);
    return f;
}

bool depends(const TT& t, int i, int k) {
    unsigned n = 1u << k;
    for (unsigned x = 0; x < n; x++)
        if (!((x >> i) & 1) && t.bit(x) != t.bit(x | (1u << i))) return true;
    return false;
}

void restrict_support(TT& t, std::vector<uint32_t>& support) {
    int k = (int)support.size();
    std::vector<int> keep;
    for (int i = 0; i < k; i++)
        if (depends(t, i, k)) keep.push_back(i);
    if ((int)keep.size() == k) return;
    int nk = (int)keep.size();
    TT nt;
    for (unsigned y = 0; y < (1u << nk); y++) {
        unsigned x = 0;
        for (int j = 0; j < nk; j++)
            if ((y >> j) & 1) x |= 1u << keep[j];
        if (t.bit(x)) nt.set(y);
    }
    std::vector<uint32_t> ns;
    for (int i : keep) ns.push_back(support[i]);
    t = nt;
    support = ns;
}

typedef std::pair<uint32_t, uint32_t> Cube;  // (care mask, value)

std::vector<Cube> prime_implicants(const TT& t, int k) {
    std::set<Cube> cur, primes;
    for (unsigned x = 0; x < (1u << k); x++)
        if (t.bit(x)) cur.insert(Cube((1u << k) - 1, x));
    while (!cur.empty()) {
        std::set<Cube> nxt, merged;
        std::vector<Cube> cl(cur.begin(), cur.end());
        for (size_t a = 0; a < cl.size(); a++)
            for (size_t b = a + 1; b < cl.size(); b++) {
                if (cl[a].first != cl[b].first) continue;
                uint32_t d = cl[a].second ^ cl[b].second;
                if (d && !(d & (d - 1))) {
                    nxt.insert(Cube(cl[a].first & ~d, cl[a].second & ~d));
                    merged.insert(cl[a]);
                    merged.insert(cl[b]);
                }
            }
        for (const Cube& c : cur)
            if (!merged.count(c)) primes.insert(c);
        cur.swap(nxt);
    }
    std::vector<Cube> out(primes.begin(), primes.end());
    std::sort(out.begin(), out.end(), [](const Cube& a, const Cube& b) {
        int pa = __builtin_popcount(a.first), pb = __builtin_popcount(b.first);
        if (pa != pb) return pa < pb;
        return a < b;
    });
    return out;
}

// Minimum cover of the true minterms (fewest terms, then fewest literals, then
// the first such combination in lexicographic index order).
std::vector<Cube> minimum_sop(const TT& t, int k) {
    std::vector<Cube> primes = prime_implicants(t, k);
    if (primes.size() > 20) return primes;
    int n = (int)primes.size();
    TT ones = t;
    std::vector<TT> cov(n);
    for (int i = 0; i < n; i++)
        for (unsigned x = 0; x < (1u << k); x++)
            if ((x & primes[i].first) == primes[i].second) cov[i].set(x);
    for (int size = 1; size <= n; size++) {
        std::vector<int> idx(size);
        for (int i = 0; i < size; i++) idx[i] = i;
        bool found = false;
        int best_lits = 0;
        std::vector<int> best;
        while (true) {
            TT s;
            int nl = 0;
            for (int i : idx) {
                s = s | cov[i];
                nl += __builtin_popcount(primes[i].first);
            }
            if ((s & ones) == ones && (!found || nl < best_lits)) {
                found = true;
                best_lits = nl;
                best = idx;
            }
            int j = size - 1;  // next combination in lexicographic order
            while (j >= 0 && idx[j] == n - size + j) j--;
            if (j < 0) break;
            idx[j]++;
            for (int q = j + 1; q < size; q++) idx[q] = idx[q - 1] + 1;
        }
        if (found) {
            std::vector<Cube> out;
            for (int i : best) out.push_back(primes[i]);
            return out;
        }
    }
    return primes;
}

// Simplified definition of var = t over support; returns false for a constant.
bool classify(uint32_t var, TT t, std::vector<uint32_t> support, Def& d) {
    restrict_support(t, support);
    int k = (int)support.size();
    if (k == 0) return false;
    d = Def();
    d.var = var;
    d.support = support;
    d.table = t;
    if (k == 1) {
        d.kind = K_LIT;
        d.lits.push_back(t.bit(1) ? (int32_t)support[0] : -(int32_t)support[0]);
        return true;
    }
    unsigned n = 1u << k;
    int ones = t.popcount();
    if (ones == 1) {
        unsigned x = 0;
        while (!t.bit(x)) x++;
        d.kind = K_AND;
        for (int i = 0; i < k; i++) d.lits.push_back(((x >> i) & 1) ? (int32_t)support[i] : -(int32_t)support[i]);
        return true;
    }
    if (ones == (int)n - 1) {
        unsigned x = 0;
        while (t.bit(x)) x++;
        d.kind = K_OR;
        for (int i = 0; i < k; i++) d.lits.push_back(((x >> i) & 1) ? -(int32_t)support[i] : (int32_t)support[i]);
        return true;
    }
    TT parity;
    for (unsigned x = 0; x < n; x++)
        if (__builtin_popcount(x) & 1) parity.set(x);
    TT full = TT::full(k);
    if (t == parity || t == parity.andnot_of(full)) {
        d.kind = K_XOR;
        d.out_neg = !(t == parity);
        for (uint32_t v : support) d.lits.push_back((int32_t)v);
        return true;
    }
    d.kind = K_SOP;
    for (const Cube& c : minimum_sop(t, k)) {
        std::vector<int32_t> term;
        for (int i = 0; i < k; i++)
            if ((c.first >> i) & 1) term.push_back(((c.second >> i) & 1) ? (int32_t)support[i] : -(int32_t)support[i]);
        d.terms.push_back(term);
    }
    return true;
}

}  // namespace

bool transform(const Cnf& cnf, const TransformOpts& o, Circuit& out, std::string& err) {
    auto t0 = std::chrono::steady_clock::now();
    if (o.max_support < 1 || o.max_support > 8) { err = "max_support must be in 1..8"; return false; }
    if (o.max_window < 1) { err = "max_window must be >= 1"; return false; }
    out = Circuit();
    out.n_vars = cnf.n_vars;
    // Clean clauses: drop repeated literals and tautologies; an empty clause is UNSAT.
    std::vector<Clause> cls;
    cls.reserve(cnf.n_clauses());
    for (size_t c = 0; c < cnf.n_clauses(); c++) {
        Clause cl;
        bool taut = false;
        for (int64_t i = cnf.off[c]; i < cnf.off[c + 1]; i++) {
            int32_t l = cnf.lits[i];
            if (std::find(cl.begin(), cl.end(), l) != cl.end()) continue;
            if (std::find(cl.begin(), cl.end(), -l) != cl.end()) taut = true;
            cl.push_back(l);
        }
        if (taut) continue;
        if (cl.empty()) { err = "empty clause: the CNF is unsatisfiable"; return false; }
        cls.push_back(std::move(cl));
    }
    if (o.reorder) {
        // key: largest variable, then longer clauses first (a variable's defining clauses
        // before unit clauses on it), then position
        std::vector<std::tuple<uint32_t, int64_t, size_t>> key(cls.size());
        for (size_t i = 0; i < cls.size(); i++) {
            uint32_t mx = 0;
            for (int32_t l : cls[i]) mx = std::max(mx, (uint32_t)std::abs(l));
            key[i] = {mx, -(int64_t)cls[i].size(), i};
        }
        std::sort(key.begin(), key.end());
        std::vector<Clause> sorted;
        sorted.reserve(cls.size());
        for (const auto& k : key) sorted.push_back(std::move(cls[std::get<2>(k)]));
        cls = std::move(sorted);
    }
    if (o.direct) {
        out.outputs = std::move(cls);
        for (uint32_t v = 1; v <= cnf.n_vars; v++) out.pis.push_back(v);
        out.wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        return true;
    }
    std::vector<int64_t> last(cnf.n_vars + 1, -1);
    for (size_t i = 0; i < cls.size(); i++)
        for (int32_t l : cls[i]) last[std::abs(l)] = (int64_t)i;
    // 0 = unclassified, 1 = primary input, 2 = intermediate
    std::vector<uint8_t> cls_of(cnf.n_vars + 1, 0);
    std::vector<size_t> SC;
    auto sc_vars = [&](const std::vector<size_t>& sc) {
        std::vector<uint32_t> vs;
        for (size_t ci : sc)
            for (int32_t l : cls[ci]) vs.push_back((uint32_t)std::abs(l));
        std::sort(vs.begin(), vs.end());
        vs.erase(std::unique(vs.begin(), vs.end()), vs.end());
        return vs;
    };
    for (size_t i = 0; i < cls.size(); i++) {
        SC.push_back(i);
        bool accepted = false;
        std::vector<uint32_t> vars = sc_vars(SC);
        for (auto it = vars.rbegin(); it != vars.rend() && !accepted; ++it) {
            uint32_t v = *it;
            if (cls_of[v] != 0) continue;
            std::vector<const Clause*> with_v;
            std::vector<size_t> without_v;
            for (size_t ci : SC) {
                bool has = false;
                for (int32_t l : cls[ci])
                    if ((uint32_t)std::abs(l) == v) has = true;
                if (has) with_v.push_back(&cls[ci]);
                else without_v.push_back(ci);
            }
            std::vector<uint32_t> support;
            for (const Clause* c : with_v)
                for (int32_t l : *c)
                    if ((uint32_t)std::abs(l) != v) support.push_back((uint32_t)std::abs(l));
            std::sort(support.begin(), support.end());
            support.erase(std::unique(support.begin(), support.end()), support.end());
            if (support.size() > o.max_support) continue;
            TT f = find_expression((int32_t)v, with_v, support);
            TT g = find_expression(-(int32_t)v, with_v, support);
            TT full = TT::full((int)support.size());
            if (f != g.andnot_of(full)) continue;
            for (size_t ci : without_v) out.outputs.push_back(cls[ci]);
            Def d;
            if (!classify(v, f, support, d)) {
                out.outputs.push_back(Clause{f == full ? (int32_t)v : -(int32_t)v});
                out.n_const++;
            } else {
                out.defs.push_back(std::move(d));
                cls_of[v] = 2;
            }
            for (uint32_t w : support)
                if (cls_of[w] != 2) cls_of[w] = 1;
            SC.clear();
            accepted = true;
        }
        if (accepted) continue;
        bool later = false;
        for (uint32_t w : vars)
            if (last[w] > (int64_t)i) { later = true; break; }
        if (!later) {
            for (size_t ci : SC) out.outputs.push_back(cls[ci]);
            SC.clear();
            continue;
        }
        while (!SC.empty() && (SC.size() > o.max_window || sc_vars(SC).size() > o.max_support)) {
            out.outputs.push_back(cls[SC.front()]);
            SC.erase(SC.begin());
        }
    }
    for (size_t ci : SC) out.outputs.push_back(cls[ci]);
    for (uint32_t v = 1; v <= cnf.n_vars; v++)
        if (cls_of[v] != 2) out.pis.push_back(v);
    out.wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return true;
}

std::string circuit_dump(const Circuit& c) {
    static const char* kn[] = {"LIT", "AND", "OR", "XOR", "SOP"};
    std::ostringstream s;
    s << "vars " << c.n_vars << "\npi";
    for (uint32_t v : c.pis) s << ' ' << v;
    s << '\n';
    for (const Def& d : c.defs) {
        s << "def " << d.var << ' ' << kn[d.kind] << ' ' << (d.out_neg ? 1 : 0) << " :";
        if (d.kind == K_SOP) {
            for (size_t t = 0; t < d.terms.size(); t++) {
                if (t) s << " |";
                for (int32_t l : d.terms[t]) s << ' ' << l;
            }
        } else {
            for (int32_t l : d.lits) s << ' ' << l;
        }
        s << '\n';
    }
    for (const auto& o : c.outputs) {
        s << "out";
        for (int32_t l : o) s << ' ' << l;
        s << '\n';
    }
    return s.str();
}

}  // namespace sat
