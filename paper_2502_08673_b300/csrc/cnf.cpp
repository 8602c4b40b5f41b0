// DIMACS CNF reader (the input format of Fig. 1(a), Section III-A).
#include <cstdlib>
#include <cstring>

#include "host.hpp"

namespace sat {

namespace {
inline bool is_space(char c) { return c == ' ' || c == '\t' || c == '\r' || c == '\n' || c == '\f' || c == '\v'; }
}  // namespace

bool parse_dimacs(const char* buf, size_t len, Cnf& out, std::string& err) {
    out = Cnf();
    const char* p = buf;
    const char* end = buf + len;
    bool have_header = false;
    uint64_t n_clauses_hdr = 0;
    bool clause_open = false;
    out.off.push_back(0);
    while (p < end) {
        while (p < end && is_space(*p)) p++;
        if (p >= end) break;
        const char* line = p;
        if (*p == 'c') {  // comment line
            while (p < end && *p != '\n') p++;
            continue;
        }
        if (*p == '%') break;  // end marker used by some benchmark files
        if (*p == 'p') {
            if (have_header) { err = "second header line"; return false; }
            const char* e = line;
            while (e < end && *e != '\n') e++;
            std::string h(line, e);
            char fmt[16] = {0};
            long long nv = -1, nc = -1;
            char extra[2] = {0};
            int got = std::sscanf(h.c_str(), "p %15s %lld %lld %1s", fmt, &nv, &nc, extra);
            if (got != 3 || std::strcmp(fmt, "cnf") != 0 || nv < 0 || nc < 0 || nv > 0x7fffffffLL) {
                err = "bad header: " + h;
                return false;
            }
            out.n_vars = (uint32_t)nv;
            n_clauses_hdr = (uint64_t)nc;
            have_header = true;
            p = e;
            continue;
        }
        if (!have_header) { err = "clause before header"; return false; }
        // one integer token
        char* q = nullptr;
        long long lit = std::strtoll(p, &q, 10);
        if (q == p || (q < end && !is_space(*q))) {
            const char* e = p;
            while (e < end && !is_space(*e)) e++;
            err = "bad token '" + std::string(p, e) + "'";
            return false;
        }
        p = q;
        if (lit == 0) {
            out.off.push_back((int64_t)out.lits.size());
            clause_open = false;
        } else {
            if (lit > (long long)out.n_vars || -lit > (long long)out.n_vars) {
                err = "literal " + std::to_string(lit) + " outside 1.." + std::to_string(out.n_vars);
                return false;
            }
            out.lits.push_back((int32_t)lit);
            clause_open = true;
        }
    }
    if (!have_header) { err = "missing header"; return false; }
    if (clause_open) { err = "last clause not terminated by 0"; return false; }
    if (out.n_clauses() != n_clauses_hdr) {
        err = "header says " + std::to_string(n_clauses_hdr) + " clauses, found " + std::to_string(out.n_clauses());
        return false;
    }
    return true;
}

}  // namespace sat
