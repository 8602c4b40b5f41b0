/* The C ABI used from plain C99 (no C++ and no Python): parse DIMACS, run Algorithm 1 on
 * the host and print what it built.  Needs no GPU.  Prints one line:
 * "<n_vars> <n_pi> <n_outputs> <n_gates> <n_cone_levels> <ops_cnf> <ops_circuit>". */
#include <stdio.h>
#include <string.h>

#include "satsampler.h"

int main(void) {
    /* Fig. 1(a) style: x3 = x1 AND x2 (Tseitin clauses), x3 must be true */
    const char* text = "p cnf 3 4\n-3 1 0\n-3 2 0\n3 -1 -2 0\n3 0\n";
    sat_cnf* cnf = NULL;
    sat_circuit* circ = NULL;
    sat_build_stats st;
    if (sat_version() == NULL) return 2;
    if (sat_cnf_from_dimacs(text, strlen(text), &cnf) != SAT_OK) {
        fprintf(stderr, "parse: %s\n", sat_last_error());
        return 3;
    }
    memset(&st, 0, sizeof st);
    if (sat_circuit_build(cnf, NULL, &circ, &st) != SAT_OK) {
        fprintf(stderr, "build: %s\n", sat_last_error());
        sat_cnf_free(cnf);
        return 4;
    }
    /* a bad argument is reported, not crashed on */
    if (sat_cnf_from_dimacs(NULL, 0, NULL) != SAT_ERR_ARG) return 5;
    printf("%u %u %u %llu %u %llu %llu\n", st.n_vars, st.n_pi, st.n_outputs, (unsigned long long)st.n_gates,
           st.n_cone_levels, (unsigned long long)st.ops_cnf, (unsigned long long)st.ops_circuit);
    sat_circuit_free(circ);
    sat_cnf_free(cnf);
    return 0;
}
