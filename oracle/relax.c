/*
 * FP64 CPU oracle for the relaxed circuit: test infrastructure only.
 *
 * Plain per-sample loops, written for checking by eye, not for speed.  Nodes
 * are evaluated in topological order; every node is one instruction
 *   y = out_neg ? 1 - h(q) : h(q),   q_i = neg_i ? 1 - p[node_i] : p[node_i]
 * with h one of (Table 1, extended to k inputs by associativity):
 *   LIT  h = q_0
 *   AND  h = prod_i q_i
 *   OR   h = 1 - prod_i (1 - q_i)
 *   XOR  h = (1 - prod_i (1 - 2 q_i)) / 2
 * Primary inputs take P = sigmoid(V) (Eq. 5); outputs feed the l2 loss of
 * Eq. 7, summed per sample in output order; the adjoint follows the chain rule
 * of Eq. 8 with the Table 1 derivatives; updates are the GD step of Eq. 9 and
 * Adam (PyTorch's formulation, no weight decay).
 *
 * Also here: Boolean evaluation of the same circuit, the CNF check against
 * the original clauses, and Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
 * with a Box-Muller transform (four normals per block) for the initial logits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OP_LIT = 0, OP_AND = 1, OP_OR = 2, OP_XOR = 3 };

typedef struct {
    int n_nodes, n_instr;
    const int *ins_out, *ins_op, *ins_neg, *ins_off, *ins_cnt; /* per instruction */
    const int *lit_node, *lit_neg;                             /* literal pool */
    int n_pi;
    const int *pi_node;                                        /* V column j -> node */
    int n_out;
    const int *out_node;
    const double *target;
} orc_circuit;

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static double lit_value(const orc_circuit *c, const double *p, int li) {
    double x = p[c->lit_node[li]];
    return c->lit_neg[li] ? 1.0 - x : x;
}

static double instr_value(const orc_circuit *c, const double *p, int k) {
    int off = c->ins_off[k], cnt = c->ins_cnt[k];
    double h, prod = 1.0;
    switch (c->ins_op[k]) {
    case OP_LIT:
        h = lit_value(c, p, off);
        break;
    case OP_AND:
        for (int i = 0; i < cnt; i++) prod *= lit_value(c, p, off + i);
        h = prod;
        break;
    case OP_OR:
        for (int i = 0; i < cnt; i++) prod *= 1.0 - lit_value(c, p, off + i);
        h = 1.0 - prod;
        break;
    default: /* XOR */
        for (int i = 0; i < cnt; i++) prod *= 1.0 - 2.0 * lit_value(c, p, off + i);
        h = 0.5 * (1.0 - prod);
        break;
    }
    return c->ins_neg[k] ? 1.0 - h : h;
}

/* dy/dq_i for instruction k (before the input literal's own negation). */
static double instr_partial(const orc_circuit *c, const double *p, int k, int i) {
    int off = c->ins_off[k], cnt = c->ins_cnt[k];
    double d = 1.0;
    switch (c->ins_op[k]) {
    case OP_LIT:
        d = 1.0;
        break;
    case OP_AND:
        for (int j = 0; j < cnt; j++) if (j != i) d *= lit_value(c, p, off + j);
        break;
    case OP_OR:
        for (int j = 0; j < cnt; j++) if (j != i) d *= 1.0 - lit_value(c, p, off + j);
        break;
    default:
        for (int j = 0; j < cnt; j++) if (j != i) d *= 1.0 - 2.0 * lit_value(c, p, off + j);
        break;
    }
    return c->ins_neg[k] ? -d : d;
}

/* V: [S][n_pi]; vals: [S][n_nodes]; loss: [S] (may be NULL). */
void orc_forward(const orc_circuit *c, int S, const double *V, double *vals, double *loss) {
#pragma omp parallel for schedule(static)
    for (int s = 0; s < S; s++) {
        double *p = vals + (size_t)s * c->n_nodes;
        for (int j = 0; j < c->n_pi; j++)
            p[c->pi_node[j]] = 1.0 / (1.0 + exp(-V[(size_t)s * c->n_pi + j]));
        for (int k = 0; k < c->n_instr; k++)
            p[c->ins_out[k]] = instr_value(c, p, k);
        if (loss) {
            double L = 0.0;
            for (int o = 0; o < c->n_out; o++) {
                double e = p[c->out_node[o]] - c->target[o];
                L += e * e;
            }
            loss[s] = L;
        }
    }
}

/* adj: [S][n_nodes] scratch (overwritten); gV: [S][n_pi] = dL/dV. */
void orc_backward(const orc_circuit *c, int S, const double *vals, double *adj, double *gV) {
#pragma omp parallel for schedule(static)
    for (int s = 0; s < S; s++) {
        const double *p = vals + (size_t)s * c->n_nodes;
        double *a = adj + (size_t)s * c->n_nodes;
        memset(a, 0, sizeof(double) * (size_t)c->n_nodes);
        for (int o = 0; o < c->n_out; o++)
            a[c->out_node[o]] += 2.0 * (p[c->out_node[o]] - c->target[o]);
        for (int k = c->n_instr - 1; k >= 0; k--) {
            double ay = a[c->ins_out[k]];
            int off = c->ins_off[k];
            for (int i = 0; i < c->ins_cnt[k]; i++) {
                double d = instr_partial(c, p, k, i);
                if (c->lit_neg[off + i]) d = -d;
                a[c->lit_node[off + i]] += ay * d;
            }
        }
        for (int j = 0; j < c->n_pi; j++) {
            double P = p[c->pi_node[j]];
            gV[(size_t)s * c->n_pi + j] = a[c->pi_node[j]] * P * (1.0 - P);
        }
    }
}

/* Magnitude of the chain rule's terms: the reverse sweep of orc_backward with every
 * fan-out term |dL/dy * dy/dx| added in absolute value, seeded with |2 (Y - T)|.
 * gVmag[s][j] = amag[pi] * P (1 - P) bounds |dL/dV| (triangle inequality), with
 * equality when no node sums terms of both signs (a single output over a fan-out-free
 * cone).  Rounding error of a floating-point adjoint is proportional to this sum of
 * absolute terms, not to the (possibly cancelled) adjoint itself: it scales tolerances. */
void orc_backward_mag(const orc_circuit *c, int S, const double *vals, double *amag, double *gVmag) {
#pragma omp parallel for schedule(static)
    for (int s = 0; s < S; s++) {
        const double *p = vals + (size_t)s * c->n_nodes;
        double *a = amag + (size_t)s * c->n_nodes;
        memset(a, 0, sizeof(double) * (size_t)c->n_nodes);
        for (int o = 0; o < c->n_out; o++)
            a[c->out_node[o]] += fabs(2.0 * (p[c->out_node[o]] - c->target[o]));
        for (int k = c->n_instr - 1; k >= 0; k--) {
            double ay = a[c->ins_out[k]];
            int off = c->ins_off[k];
            for (int i = 0; i < c->ins_cnt[k]; i++)
                a[c->lit_node[off + i]] += ay * fabs(instr_partial(c, p, k, i));
        }
        for (int j = 0; j < c->n_pi; j++) {
            double P = p[c->pi_node[j]];
            gVmag[(size_t)s * c->n_pi + j] = a[c->pi_node[j]] * P * (1.0 - P);
        }
    }
}

void orc_gd(long n, double *V, const double *g, double lr) {
    for (long i = 0; i < n; i++) V[i] -= lr * g[i];
}

/* One Adam step at step count t >= 1. */
void orc_adam(long n, double *V, double *m, double *v, const double *g, int t,
              double lr, double b1, double b2, double eps) {
    double bc1 = 1.0 - pow(b1, t), bc2 = 1.0 - pow(b2, t);
    for (long i = 0; i < n; i++) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        V[i] -= lr * (m[i] / bc1) / (sqrt(v[i] / bc2) + eps);
    }
}

/* Boolean evaluation: pi_bits [S][n_pi], bits [S][n_nodes] (0/1 bytes). */
void orc_hard(const orc_circuit *c, int S, const unsigned char *pi_bits, unsigned char *bits) {
#pragma omp parallel for schedule(static)
    for (int s = 0; s < S; s++) {
        unsigned char *b = bits + (size_t)s * c->n_nodes;
        for (int j = 0; j < c->n_pi; j++) b[c->pi_node[j]] = pi_bits[(size_t)s * c->n_pi + j];
        for (int k = 0; k < c->n_instr; k++) {
            int off = c->ins_off[k], cnt = c->ins_cnt[k], y;
            switch (c->ins_op[k]) {
            case OP_LIT: y = b[c->lit_node[off]] ^ c->lit_neg[off]; break;
            case OP_AND: y = 1; for (int i = 0; i < cnt; i++) y &= b[c->lit_node[off + i]] ^ c->lit_neg[off + i]; break;
            case OP_OR:  y = 0; for (int i = 0; i < cnt; i++) y |= b[c->lit_node[off + i]] ^ c->lit_neg[off + i]; break;
            default:     y = 0; for (int i = 0; i < cnt; i++) y ^= b[c->lit_node[off + i]] ^ c->lit_neg[off + i]; break;
            }
            b[c->ins_out[k]] = (unsigned char)(y ^ c->ins_neg[k]);
        }
    }
}

/* CNF check on full assignments assign [S][n_vars+1] (index 0 unused). */
void orc_cnf_check(int n_clauses, const long *off, const int *lits, int n_vars, int S,
                   const unsigned char *assign, unsigned char *ok) {
#pragma omp parallel for schedule(static)
    for (int s = 0; s < S; s++) {
        const unsigned char *x = assign + (size_t)s * (n_vars + 1);
        int good = 1;
        for (int ci = 0; ci < n_clauses && good; ci++) {
            int sat = 0;
            for (long i = off[ci]; i < off[ci + 1]; i++) {
                int l = lits[i];
                if ((l > 0 && x[l]) || (l < 0 && !x[-l])) { sat = 1; break; }
            }
            good = sat;
        }
        ok[s] = (unsigned char)good;
    }
}

/* Philox4x32-10 block function (SC'11, Section 4). */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Initial logits V0[s][j] = scale * z_k, k = s mod 4: the Philox block of counter
 * (s / 4, j, round, 0) under key (seed lo, seed hi) gives four normals, the Box-Muller
 * pairs (cos, sin) of its words (0, 1) and (2, 3). */
void orc_init_normal(int S, int n_pi, uint64_t seed, uint32_t round, double scale, double *V) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int s = 0; s < S; s++)
        for (int j = 0; j < n_pi; j++) {
            uint32_t ctr[4] = {(uint32_t)(s / 4), (uint32_t)j, round, 0u}, o[4];
            orc_philox4x32_10(ctr, key, o);
            int k = s % 4;
            uint32_t a = o[k < 2 ? 0 : 2], b = o[k < 2 ? 1 : 3];
            double u1 = (double)((a >> 8) + 1u) * (1.0 / 16777216.0);
            double u2 = (double)(b >> 8) * (1.0 / 16777216.0);
            double rad = sqrt(-2.0 * log(u1));
            V[(size_t)s * n_pi + j] = scale * rad * ((k % 2 == 0) ? cos(2.0 * M_PI * u2) : sin(2.0 * M_PI * u2));
        }
}
