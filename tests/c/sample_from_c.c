/* End to end from plain C99 on the GPU: sat_cnf_from_file -> sat_circuit_build ->
 * sat_sample -> sat_solutions_copy.  Usage: sample_from_c <in.cnf> <out.txt>.  Writes the
 * number of variables and solutions, then one line of hex words per solution. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "satsampler.h"

int main(int argc, char** argv) {
    sat_cnf* cnf = NULL;
    sat_circuit* circ = NULL;
    sat_solutions* sols = NULL;
    sat_sample_opts o;
    sat_sample_stats st;
    sat_status s;
    uint64_t n, i, w, nw;
    uint64_t* words;
    FILE* f;
    if (argc != 3) return 2;
    if (sat_cnf_from_file(argv[1], &cnf) != SAT_OK || sat_circuit_build(cnf, NULL, &circ, NULL) != SAT_OK) {
        fprintf(stderr, "%s\n", sat_last_error());
        return 3;
    }
    sat_sample_opts_default(&o);
    o.batch = 1024;
    o.steps = 200;
    o.max_rounds = 2;
    s = sat_sample(circ, cnf, &o, 1000000, &sols, &st);
    if (s != SAT_OK && s != SAT_PARTIAL) {
        fprintf(stderr, "sample: %s\n", sat_last_error());
        return 4;
    }
    n = sat_solutions_count(sols);
    nw = (sat_solutions_nvars(sols) + 63) / 64;
    words = (uint64_t*)malloc((n ? n : 1) * nw * sizeof(uint64_t));
    if (!words || sat_solutions_copy(sols, 0, n, words) != SAT_OK) return 5;
    f = fopen(argv[2], "w");
    if (!f) return 6;
    fprintf(f, "%u %llu\n", sat_solutions_nvars(sols), (unsigned long long)n);
    for (i = 0; i < n; i++) {
        for (w = 0; w < nw; w++) fprintf(f, "%016llx%s", (unsigned long long)words[i * nw + w], w + 1 < nw ? " " : "\n");
    }
    fclose(f);
    free(words);
    sat_solutions_free(sols);
    sat_circuit_free(circ);
    sat_cnf_free(cnf);
    return 0;
}
