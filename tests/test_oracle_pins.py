"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names what it pins: worked examples printed in the paper (Fig. 1,
Eq. c1, Eqs. 1-4, Table 1), exhaustive enumeration on small instances, central
finite differences, closed forms of the optimiser steps, and published
known-answer vectors of Philox4x32-10 and SplitMix64.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import transform as fz
from oracle.dimacs import parse_dimacs, DimacsError, cnf_satisfied
from workloads import tseitin_random_circuit, planted_3sat, fig1_example_dimacs, dimacs_text


# ---------------------------------------------------------------- Fig. 1 ----
def test_fig1_transformation():
    """Fig. 1(a)-(c): PIs {x1,x6,x11,x12,x13,x14}, aliases x2..x4, x7..x9, MUXes x5, x10, PO x10 = 1."""
    n, cl = parse_dimacs(fig1_example_dimacs())
    assert (n, len(cl)) == (14, 21)
    c = fz.factorize(n, cl)
    assert c.pis == [1, 6, 11, 12, 13, 14]
    d = {x.var: x for x in c.defs}
    assert sorted(d) == [2, 3, 4, 5, 7, 8, 9, 10]
    assert (d[2].kind, d[2].lits) == ("LIT", [-1])
    assert (d[3].kind, d[3].lits) == ("LIT", [2])
    assert (d[4].kind, d[4].lits) == ("LIT", [3])
    assert (d[9].kind, d[9].lits) == ("LIT", [-8])
    # Fig. 1(c) relaxes x5 = OR(AND(x4, x11), AND(NOT(x4), x12)), likewise x10.
    assert (d[5].kind, d[5].lits) == ("SOP", [[4, 11], [-4, 12]])
    assert (d[10].kind, d[10].lits) == ("SOP", [[9, 13], [-9, 14]])
    assert c.outputs == [[10]]


def _count_cnf(n, cl):
    sols = set()
    for bits in itertools.product([0, 1], repeat=n):
        a = (0,) + bits
        if cnf_satisfied(cl, a):
            sols.add(bits)
    return sols


def _count_circuit(c):
    sols = set()
    for bits in itertools.product([0, 1], repeat=len(c.pis)):
        val = fz.circuit_assignment(c, dict(zip(c.pis, bits)))
        if fz.outputs_satisfied(c, val):
            sols.add(tuple(val[v] for v in range(1, c.n_vars + 1)))
    return sols


def test_fig1_solution_count():
    """#SAT of Fig. 1(a) is 32 in CNF space and in PI space, with the same solution set."""
    n, cl = parse_dimacs(fig1_example_dimacs())
    cnf = _count_cnf(n, cl)
    circ = _count_circuit(fz.factorize(n, cl))
    assert len(cnf) == 32
    assert circ == cnf


# --------------------------------------------------------- Eq. c1 / MUX ----
def test_mux_complement_check():
    """Eq. c1: x5 = (x107 AND x4) OR (x108 AND NOT x4) is found; x4, x107, x108 are not definable."""
    SC = [[-4, -107, 5], [-4, 107, -5], [4, -108, 5], [4, 108, -5]]
    sup = [4, 107, 108]
    f = fz.find_boolean_expression(5, SC, sup)
    g = fz.find_boolean_expression(-5, SC, sup)
    expect = 0
    for x in range(8):
        x4, x107, x108 = x & 1, (x >> 1) & 1, (x >> 2) & 1
        if (x107 and x4) or (x108 and not x4):
            expect |= 1 << x
    assert f == expect
    assert g == (~expect & 0xFF)       # the paper's complementary expression
    for v in (4, 107, 108):
        s = sorted({abs(l) for c in SC for l in c} - {v})
        fv = fz.find_boolean_expression(v, SC, s)
        gv = fz.find_boolean_expression(-v, SC, s)
        assert fv != (~gv & ((1 << (1 << len(s))) - 1))
    c = fz.factorize(108, SC)
    assert [(d.var, d.kind) for d in c.defs] == [(5, "SOP")]
    assert c.outputs == []


# ------------------------------------------------------ Eqs. 1-4 signatures -
def _sig_clauses(kind, n):
    f = n + 1
    xs = list(range(1, n + 1))
    if kind == "NOT":
        return [[f, 1], [-f, -1]]
    if kind in ("OR", "NOR"):
        s = 1 if kind == "OR" else -1
        return [[-s * f] + xs] + [[s * f, -x] for x in xs]
    if kind in ("AND", "NAND"):
        s = 1 if kind == "AND" else -1
        return [[s * f] + [-x for x in xs]] + [[-s * f, x] for x in xs]
    # XOR / XNOR of n inputs: forbid every assignment of (x, f) with the wrong parity
    out = []
    for bits in itertools.product([0, 1], repeat=n + 1):
        par = sum(bits[:n]) & 1
        want = par if kind == "XOR" else 1 - par
        if bits[n] != want:
            out.append([-(i + 1) if b else (i + 1) for i, b in enumerate(bits)])
    return out


@pytest.mark.parametrize("kind,n", [("NOT", 1), ("OR", 2), ("OR", 3), ("AND", 2), ("AND", 4),
                                    ("NAND", 3), ("NOR", 2), ("XOR", 2), ("XOR", 3), ("XNOR", 2), ("XNOR", 3)])
def test_cnf_signatures(kind, n):
    """Eqs. 1-4: each signature is recognised as its gate, in every clause order."""
    base = _sig_clauses(kind, n)
    f = n + 1
    for perm in list(itertools.permutations(base))[:24]:
        c = fz.factorize(n + 1, list(perm))
        assert c.outputs == []
        (d,) = c.defs
        assert d.var == f
        val_fn = {
            "NOT": lambda x: 1 - x[0], "OR": lambda x: int(any(x)), "NOR": lambda x: 1 - int(any(x)),
            "AND": lambda x: int(all(x)), "NAND": lambda x: 1 - int(all(x)),
            "XOR": lambda x: sum(x) & 1, "XNOR": lambda x: 1 - (sum(x) & 1)}[kind]
        for bits in itertools.product([0, 1], repeat=n):
            val = fz.circuit_assignment(c, dict(zip(range(1, n + 1), bits)))
            assert val[f] == val_fn(bits)
        # NAND/NOR are recognised in De Morgan form (OR/AND of negated literals):
        # the same function, and the same relaxation (1 - prod p_i, resp. prod (1 - p_i)).
        expect_kind = {"NOT": "LIT", "OR": "OR", "NOR": "AND", "AND": "AND", "NAND": "OR",
                       "XOR": "XOR", "XNOR": "XOR"}[kind]
        assert d.kind == expect_kind


# ------------------------------------------------------ exhaustive checks ---
@pytest.mark.parametrize("seed", range(6))
def test_small_tseitin_bruteforce(seed):
    """CNF-space and PI-space enumeration agree (count and full solution sets)."""
    inst = tseitin_random_circuit(n_pi=6, n_gates=12, depth=4, n_out=2, seed=seed)
    n, cl = parse_dimacs(inst.dimacs())
    assert n == 18
    c = fz.factorize(n, cl)
    assert _count_circuit(c) == _count_cnf(n, cl)


@pytest.mark.parametrize("seed", range(4))
def test_small_planted3sat_bruteforce(seed):
    inst = planted_3sat(14, 50, seed)
    n, cl = parse_dimacs(inst.dimacs())
    c = fz.factorize(n, cl)
    sols = _count_circuit(c)
    assert sols == _count_cnf(n, cl)
    assert tuple(int(x) for x in inst.hidden) in sols


@pytest.mark.parametrize("seed", range(3))
def test_reorder_shuffled_tseitin_bruteforce(seed):
    """Clauses shuffled, then reordered: the solution set is still the CNF's (enumeration in
    both spaces) and every generated gate is recovered as an intermediate variable."""
    import random
    inst = tseitin_random_circuit(n_pi=6, n_gates=12, depth=4, n_out=2, seed=seed)
    n, cl = parse_dimacs(inst.dimacs())
    sh = random.Random(seed + 10).sample(cl, len(cl))
    c = fz.factorize(n, sh, reorder=True)
    assert c.pis == list(range(1, 7)) and sorted(d.var for d in c.defs) == list(range(7, 19))
    assert _count_circuit(c) == _count_cnf(n, sh)


@pytest.mark.parametrize("seed", range(3))
def test_direct_circuit_bruteforce(seed):
    """Direct relaxation (no factorization): every variable an input, every clause an
    OR output; its solutions are the CNF's, and its flattened gates, evaluated on
    every assignment, are all 1 exactly where the CNF holds."""
    n, cl = parse_dimacs(planted_3sat(12, 45, seed).dimacs())
    cl = cl + [[1, -1, 3]]  # plus a tautology, which is dropped
    c = fz.direct_circuit(n, cl)
    assert c.pis == list(range(1, n + 1)) and c.defs == [] and len(c.outputs) == 45
    assert _count_circuit(c) == _count_cnf(n, cl)
    fc = oracle.flatten(c)
    allb = np.array(list(itertools.product([0, 1], repeat=n)), dtype=np.uint8)
    bits = oracle.hard_eval(fc, allb)
    outs_ok = (bits[:, fc.out_node] == fc.target[None, :]).all(axis=1)
    assign = np.zeros((len(allb), n + 1), np.uint8)
    assign[:, 1:] = allb
    assert (outs_ok == oracle.cnf_check(n, cl, assign).astype(bool)).all()


def test_tseitin_ground_truth_gates():
    """Every generated gate is recovered with the generator's Boolean function."""
    inst = tseitin_random_circuit(n_pi=40, n_gates=120, depth=6, n_out=4, seed=3)
    n, cl = parse_dimacs(inst.dimacs())
    c = fz.factorize(n, cl)
    assert c.pis == list(range(1, 41))
    assert [d.var for d in c.defs] == list(range(41, 161))
    rng = np.random.default_rng(0)
    pis = rng.integers(0, 2, (64, 40)).astype(np.uint8)
    truth = inst.ground_truth_values(pis)
    for s in range(64):
        val = fz.circuit_assignment(c, {v: int(pis[s, v - 1]) for v in c.pis})
        assert [val[v] for v in range(1, n + 1)] == list(truth[s])
    assert sorted(map(tuple, c.outputs)) == sorted(
        ((int(o) + 1) if t else -(int(o) + 1),) for o, t in zip(inst.out_nodes, inst.targets))


# ---------------------------------------------------------------- Table 1 ---
def _one_gate(kind, out_neg=False):
    defs = [fz.Definition(3, kind, [1, 2], out_neg)]
    return oracle.flatten(fz.Circuit(3, [1, 2], defs, [[3]]))


def _P(p):
    return np.log(p) - np.log1p(-p)  # logit


@pytest.mark.parametrize("kind,formula,d1,d2", [
    ("AND", lambda a, b: a * b, lambda a, b: b, lambda a, b: a),
    ("OR", lambda a, b: 1 - (1 - a) * (1 - b), lambda a, b: 1 - b, lambda a, b: 1 - a),
    ("XOR", lambda a, b: (1 - a) * b + a * (1 - b), lambda a, b: 1 - 2 * b, lambda a, b: 1 - 2 * a),
])
def test_table1_values_and_derivatives(kind, formula, d1, d2):
    """Table 1 closed forms (as printed) for gate values and input derivatives."""
    fc = _one_gate(kind)
    rng = np.random.default_rng(1)
    P = rng.uniform(0.02, 0.98, (50, 2))
    vals, loss = oracle.forward(fc, _P(P))
    a, b = P[:, 0], P[:, 1]
    y = formula(a, b)
    np.testing.assert_allclose(vals[:, 2], y, rtol=0, atol=1e-13)
    np.testing.assert_allclose(loss, (y - 1) ** 2, atol=1e-13)
    gV, adj = oracle.backward(fc, vals)
    np.testing.assert_allclose(adj[:, 0], 2 * (y - 1) * d1(a, b), atol=1e-12)
    np.testing.assert_allclose(adj[:, 1], 2 * (y - 1) * d2(a, b), atol=1e-12)
    np.testing.assert_allclose(gV[:, 0], adj[:, 0] * a * (1 - a), atol=1e-12)


def test_table1_xnor_not():
    fc = _one_gate("XOR", out_neg=True)
    P = np.array([[0.3, 0.8], [0.9, 0.1]])
    vals, _ = oracle.forward(fc, _P(P))
    a, b = P[:, 0], P[:, 1]
    np.testing.assert_allclose(vals[:, 2], a * b + (1 - a) * (1 - b), atol=1e-13)
    gV, adj = oracle.backward(fc, vals)
    y = vals[:, 2]
    np.testing.assert_allclose(adj[:, 0], 2 * (y - 1) * (2 * b - 1), atol=1e-12)
    fcn = oracle.flatten(fz.Circuit(2, [1], [fz.Definition(2, "LIT", [-1])], [[2]]))
    vals, _ = oracle.forward(fcn, _P(np.array([[0.25]])))
    assert abs(vals[0, 1] - 0.75) < 1e-14
    gV, adj = oracle.backward(fcn, vals)
    assert abs(adj[0, 0] - 2 * (0.75 - 1) * (-1)) < 1e-14


def test_vertex_invariant():
    """On {0,1} inputs the relaxation equals the Boolean circuit exactly (every node)."""
    inst = tseitin_random_circuit(n_pi=30, n_gates=90, depth=6, n_out=3, seed=5)
    o = oracle.Oracle(inst.dimacs())
    rng = np.random.default_rng(2)
    bits = rng.integers(0, 2, (40, o.n_pi)).astype(np.uint8)
    V = np.where(bits == 1, np.inf, -np.inf)
    vals, _ = oracle.forward(o.flat, V)
    hard = oracle.hard_eval(o.flat, bits)
    np.testing.assert_array_equal(vals, hard.astype(np.float64))


def test_fig1_sop_matches_figure_relaxation():
    """Fig. 1(c): x10 = OR(AND(x9,x13), AND(NOT x9,x14)) with x9 = NOT(x6)."""
    o = oracle.Oracle(fig1_example_dimacs())
    rng = np.random.default_rng(4)
    V = rng.normal(size=(20, o.n_pi))
    vals, loss = oracle.forward(o.flat, V)
    P = 1 / (1 + np.exp(-V))
    pi = dict(zip(o.circuit.pis, P.T))
    x9 = 1 - pi[6]
    x10 = 1 - (1 - x9 * pi[13]) * (1 - (1 - x9) * pi[14])
    np.testing.assert_allclose(vals[:, 9], x10, atol=1e-14)
    np.testing.assert_allclose(loss, (x10 - 1) ** 2, atol=1e-14)
    # the chain rule of Eq. 8 with Table 1 derivatives (not the garbled printed form)
    gV, adj = oracle.backward(o.flat, vals)
    np.testing.assert_allclose(adj[:, 12], 2 * (x10 - 1) * x9 * (1 - (1 - x9) * pi[14]), atol=1e-13)


# --------------------------------------------------- finite differences ----
@pytest.mark.parametrize("seed", range(3))
def test_gradient_central_differences(seed):
    """dL/dV against central differences in FP64: relative error <= 1e-6."""
    inst = tseitin_random_circuit(n_pi=20, n_gates=60, depth=6, n_out=4, seed=seed)
    o = oracle.Oracle(inst.dimacs())
    rng = np.random.default_rng(seed)
    V = rng.normal(size=(4, o.n_pi))
    vals, loss = oracle.forward(o.flat, V)
    gV, _ = oracle.backward(o.flat, vals)
    h = 1e-5
    fd = np.zeros_like(V)
    for j in range(o.n_pi):
        Vp, Vm = V.copy(), V.copy()
        Vp[:, j] += h
        Vm[:, j] -= h
        fd[:, j] = (oracle.forward(o.flat, Vp)[1] - oracle.forward(o.flat, Vm)[1]) / (2 * h)
    scale = np.abs(gV).max(axis=1, keepdims=True)
    assert (scale > 1e-6).all()
    assert (np.abs(fd - gV) <= 1e-6 * scale).all()


def test_gradient_fd_sop_and_wide_gates():
    """Same check through SOP definitions (Fig. 1) and 3-input OR outputs (3-SAT)."""
    for text in (fig1_example_dimacs(), planted_3sat(12, 30, 7).dimacs()):
        o = oracle.Oracle(text)
        rng = np.random.default_rng(9)
        V = rng.normal(size=(3, o.n_pi))
        gV, _ = oracle.backward(o.flat, oracle.forward(o.flat, V)[0])
        h = 1e-5
        for j in range(o.n_pi):
            Vp, Vm = V.copy(), V.copy()
            Vp[:, j] += h
            Vm[:, j] -= h
            fd = (oracle.forward(o.flat, Vp)[1] - oracle.forward(o.flat, Vm)[1]) / (2 * h)
            assert np.all(np.abs(fd - gV[:, j]) <= 1e-6 * np.abs(gV).max(axis=1) + 1e-12)


# ------------------------------------------- magnitude of the chain rule ----
def _gate_clauses(y, a, b, op):
    """CNF of y = op(a, b) for literals a, b (the signatures of Eqs. 1-3)."""
    if op == "and":
        return [[-y, a], [-y, b], [y, -a, -b]]
    if op == "or":
        return [[y, -a], [y, -b], [-y, a, b]]
    return [[-y, a, b], [-y, -a, -b], [y, -a, b], [y, a, -b]]


# Two fan-out-free trees over inputs 1..8 that share input 1:
# 9 = AND(1, -2), 10 = XOR(3, 4), 11 = OR(9, 10)  (tree 1, output 11)
# 12 = OR(-1, 5), 13 = XOR(6, -7), 14 = AND(12, -13), 15 = XOR(14, 8)  (tree 2, output 15)
_TREES = [(9, 1, -2, "and"), (10, 3, 4, "xor"), (11, 9, 10, "or"),
          (12, -1, 5, "or"), (13, 6, -7, "xor"), (14, 12, -13, "and"), (15, 14, 8, "xor")]


def _tree_oracle(outputs):
    clauses = [c for g in _TREES for c in _gate_clauses(*g)] + [[o] for o in outputs]
    return oracle.Oracle(dimacs_text(15, clauses))


def test_gradient_magnitude_bounds_gradient():
    """sum_terms |.| >= |dL/dV| on circuits with reconvergent fan-out and many outputs."""
    for text in (tseitin_random_circuit(40, 200, 8, 6, seed=2).dimacs(), planted_3sat(20, 60, 3).dimacs(),
                 fig1_example_dimacs()):
        o = oracle.Oracle(text)
        V = np.random.default_rng(4).normal(size=(5, o.n_pi))
        vals, _ = oracle.forward(o.flat, V)
        g, _ = oracle.backward(o.flat, vals)
        gm = oracle.backward_magnitude(o.flat, vals)
        assert (gm >= np.abs(g) * (1 - 1e-12)).all()
        assert (gm > np.abs(g) * (1 + 1e-9)).any()  # some input sums terms of both signs


def test_gradient_magnitude_on_trees():
    """A single output over a fan-out-free cone has one term per adjoint: magnitude = |dL/dV|.
    Two outputs whose trees share input 1: at input 1 the magnitude is the sum of the two
    single-output gradients' absolute values, while the gradient is their signed sum."""
    V = np.random.default_rng(6).normal(size=(7, 8))
    single = {}
    for out in (11, 15):
        o = _tree_oracle([out])
        assert o.circuit.pis == list(range(1, 9))
        vals, _ = oracle.forward(o.flat, V)
        g, _ = oracle.backward(o.flat, vals)
        gm = oracle.backward_magnitude(o.flat, vals)
        np.testing.assert_allclose(gm, np.abs(g), rtol=1e-13, atol=0)
        single[out] = g
    o = _tree_oracle([11, 15])
    vals, _ = oracle.forward(o.flat, V)
    g, _ = oracle.backward(o.flat, vals)
    gm = oracle.backward_magnitude(o.flat, vals)
    np.testing.assert_allclose(g, single[11] + single[15], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(gm[:, 0], np.abs(single[11][:, 0]) + np.abs(single[15][:, 0]), rtol=1e-13)
    np.testing.assert_allclose(gm[:, 1:], np.abs(g[:, 1:]), rtol=1e-13, atol=0)


# -------------------------------------------------------------- optimisers -
def test_adam_first_step_closed_form():
    """Adam at t=1: m_hat = g, v_hat = g^2, so V1 = V0 - lr * g / (|g| + eps)."""
    rng = np.random.default_rng(0)
    V0 = rng.normal(size=100)
    g = rng.normal(size=100) * 10.0 ** rng.uniform(-6, 2, 100)
    V, m, v = V0.copy(), np.zeros(100), np.zeros(100)
    oracle.adam_step(V, m, v, g, 1, 0.1)
    np.testing.assert_allclose(V, V0 - 0.1 * g / (np.abs(g) + 1e-8), rtol=1e-14, atol=1e-15)


def test_adam_second_step_closed_form():
    """t=2 with beta1=0.9, beta2=0.999 written out from the bias-corrected moments."""
    g1, g2, lr = 0.3, -0.7, 0.05
    V, m, v = np.array([1.0]), np.zeros(1), np.zeros(1)
    oracle.adam_step(V, m, v, np.array([g1]), 1, lr)
    oracle.adam_step(V, m, v, np.array([g2]), 2, lr)
    m2 = 0.9 * 0.1 * g1 + 0.1 * g2
    v2 = 0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2
    step1 = lr * g1 / (abs(g1) + 1e-8)
    step2 = lr * (m2 / (1 - 0.81)) / (math.sqrt(v2 / (1 - 0.999 ** 2)) + 1e-8)
    assert abs(V[0] - (1.0 - step1 - step2)) < 1e-14


def test_gd_step():
    """Eq. 9 exactly."""
    V = np.array([1.0, -2.0])
    oracle.gd_step(V, np.array([0.5, 0.25]), 10.0)
    assert list(V) == [-4.0, -4.5]


def test_planted_fixed_point():
    """Started at the planted input (|V0| = 30), the round returns exactly that solution."""
    inst = tseitin_random_circuit(n_pi=50, n_gates=300, depth=10, n_out=8, seed=11)
    o = oracle.Oracle(inst.dimacs())
    V0 = np.where(inst.planted[None, :] == 1, 30.0, -30.0).repeat(4, axis=0)
    vals, loss = oracle.forward(o.flat, V0)
    assert loss.max() < 1e-20
    res = oracle.sample_round(o.flat, o.n_vars, o.clauses, V0, steps=20, lr=0.1)
    assert res["valid"].all()
    assert len(res["unique"]) == 1
    (key,) = res["unique"]
    truth = inst.ground_truth_values(inst.planted[None, :])[0]
    assert key == truth.tobytes()


# ------------------------------------------------------- verification -----
def test_cnf_check_matches_enumeration():
    inst = planted_3sat(10, 40, 3)
    n, cl = parse_dimacs(inst.dimacs())
    allb = np.array(list(itertools.product([0, 1], repeat=n)), dtype=np.uint8)
    assign = np.zeros((len(allb), n + 1), np.uint8)
    assign[:, 1:] = allb
    ok = oracle.cnf_check(n, cl, assign)
    expect = [cnf_satisfied(cl, (0,) + tuple(r)) for r in allb]
    assert list(ok.astype(bool)) == expect


def test_philox_known_answers():
    """Known-answer vectors of Philox4x32-10 (Random123 distribution, SC'11)."""
    assert oracle.philox4x32_10([0, 0, 0, 0], [0, 0]) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    assert oracle.philox4x32_10([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2) == [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    assert oracle.philox4x32_10([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0]) == \
        [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_init_normal_uses_the_stated_blocks():
    """V0[s][j] = scale z_(s mod 4) from the Philox block of counter (s // 4, j, round, 0): entries
    re-derived from the pinned block function, and the pair structure of Box-Muller (the two
    normals of a pair are uncorrelated; z0^2 + z1^2 is exponential with mean 2)."""
    V = oracle.init_normal(4001, 7, seed=0x1234_5678_9ABC, rnd=3, scale=1.5)
    key = [0x5678_9ABC, 0x1234]
    for s, j in ((0, 0), (5, 3), (10, 6), (4000, 2)):
        o = oracle.philox4x32_10([s // 4, j, 3, 0], key)
        k = s % 4
        a, b = (o[0], o[1]) if k < 2 else (o[2], o[3])
        r = math.sqrt(-2 * math.log(((a >> 8) + 1) / 2 ** 24))
        t = 2 * math.pi * (b >> 8) / 2 ** 24
        assert abs(V[s, j] - 1.5 * r * (math.cos(t) if k % 2 == 0 else math.sin(t))) < 1e-12
    Z = oracle.init_normal(40000, 4, seed=9, rnd=0, scale=1.0)
    z0, z1 = Z[0::4].ravel(), Z[1::4].ravel()
    assert abs(np.corrcoef(z0, z1)[0, 1]) < 0.02
    assert abs((z0 ** 2 + z1 ** 2).mean() - 2.0) < 0.05 and abs(np.median(z0 ** 2 + z1 ** 2) - 2 * math.log(2)) < 0.05


def test_init_normal_moments():
    V = oracle.init_normal(4000, 16, seed=5, rnd=0, scale=2.0)
    assert abs(V.mean()) < 0.05 and abs(V.std() - 2.0) < 0.05
    assert np.array_equal(V, oracle.init_normal(4000, 16, seed=5, rnd=0, scale=2.0))
    assert not np.array_equal(V, oracle.init_normal(4000, 16, seed=5, rnd=1, scale=2.0))


def test_splitmix64_finaliser():
    """SplitMix64 seeded with 0 yields 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4 (Steele et al. 2014)."""
    from oracle.sampler import _mix64
    gamma = 0x9E3779B97F4A7C15
    assert _mix64(gamma) == 0xE220A8397B1DCDAF
    assert _mix64((2 * gamma) & ((1 << 64) - 1)) == 0x6E789E6AA1B965F4


def test_dedup_is_set_semantics():
    inst = tseitin_random_circuit(n_pi=12, n_gates=24, depth=4, n_out=1, seed=2)
    o = oracle.Oracle(inst.dimacs())
    rng = np.random.default_rng(0)
    V = rng.choice([-1.0, 1.0], size=(300, o.n_pi))
    res = oracle.verify(o.flat, o.n_vars, o.clauses, V)
    keys = {res["assign"][s, 1:].tobytes() for s in range(300) if res["valid"][s]}
    assert set(res["unique"]) == keys
    assert 0 < len(keys) < 300


# --------------------------------------------------------------- parsing ---
@pytest.mark.parametrize("text", [
    "p cnf 3 2\n1 2 0\n", "p cnf 2 1\n1 3 0\n", "1 2 0\n", "p cnf 2 1\n1 2\n", "p cnf x 1\n1 0\n",
])
def test_dimacs_errors(text):
    with pytest.raises(DimacsError):
        parse_dimacs(text)


def test_dimacs_multiline_and_comments():
    n, cl = parse_dimacs("c hi\np cnf 3 2\n1 -2\n 3 0 -1\n0\n%\n0\n")
    assert n == 3 and cl == [[1, -2, 3], [-1]]
