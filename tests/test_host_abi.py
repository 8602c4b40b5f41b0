"""CPU tests of the library's host side: the C ABI loads and exports every
declared symbol, the DIMACS reader's errors, and the native transformation
(Algorithm 1) against the oracle's, bit-exact in canonical form."""
import ctypes

import pytest

import oracle
from oracle import transform as fz
from oracle.dimacs import parse_dimacs
from workloads import tseitin_random_circuit, planted_3sat, fig1_example_dimacs, dimacs_text
from tests.helpers import oracle_dump, header_functions

import paper_2502_08673_b300 as P
from paper_2502_08673_b300 import _native


def test_library_exports_every_declared_symbol():
    names = header_functions()
    assert len(names) >= 30
    lib = ctypes.CDLL(str(_native.LIB_PATH))
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) <= set(_native.PROTOTYPES), set(names) - set(_native.PROTOTYPES)


def _native_dump(text):
    return P.Circuit.build(P.Cnf.from_dimacs(text)).dump()


def _oracle_dump(text):
    n, cl = parse_dimacs(text)
    return oracle_dump(fz.factorize(n, cl))


def test_reorder_build_matches_oracle_and_recovers_shuffled_gates():
    """reorder=True: the native build equals the oracle's on shuffled clauses, and a
    shuffled Tseitin file yields the same circuit as the file in gate order."""
    import random
    n, cl = parse_dimacs(tseitin_random_circuit(40, 160, 8, 4, seed=2).dimacs())
    base = oracle_dump(fz.factorize(n, cl))
    for seed in range(3):
        sh = random.Random(seed).sample(cl, len(cl))
        text = dimacs_text(n, sh)
        native = P.Circuit.build(P.Cnf.from_dimacs(text), reorder=True).dump()
        assert native == oracle_dump(fz.factorize(n, sh, reorder=True))
        assert native == base
    n3, cl3 = parse_dimacs(planted_3sat(30, 120, 2).dimacs())
    text3 = dimacs_text(n3, cl3[::-1])
    assert P.Circuit.build(P.Cnf.from_dimacs(text3), reorder=True).dump() == \
        oracle_dump(fz.factorize(n3, cl3[::-1], reorder=True))


def test_direct_build_matches_oracle():
    """direct=True: the cleaned clauses as outputs, all variables as inputs."""
    n0, cl0 = parse_dimacs(planted_3sat(30, 120, 5).dimacs())
    with_extras = dimacs_text(n0, cl0 + [[2, -2, 7], [3, 3, -4]])  # a tautology and a repeated literal
    for text in (with_extras, tseitin_random_circuit(20, 60, 6, 3, seed=1).dimacs()):
        circ = P.Circuit.build(P.Cnf.from_dimacs(text), direct=True)
        n, cl = parse_dimacs(text)
        assert circ.dump() == oracle_dump(fz.direct_circuit(n, cl))
        st = circ.stats
        assert st["n_pi"] == n and st["n_iv"] == 0 and st["n_outputs"] == len(fz.direct_circuit(n, cl).outputs)


CASES = {
    "fig1": fig1_example_dimacs,
    "tseitin_small": lambda: tseitin_random_circuit(20, 60, 6, 3, seed=1).dimacs(),
    "tseitin_c1size": lambda: tseitin_random_circuit(200, 2000, 20, 16, seed=2).dimacs(),
    "planted3sat_c1": lambda: planted_3sat(50, 200, 1).dimacs(),
    "planted3sat_dense": lambda: planted_3sat(30, 200, 4).dimacs(),
    "mux_window": lambda: dimacs_text(108, [[-4, -107, 5], [-4, 107, -5], [4, -108, 5], [4, 108, -5]]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_transform_matches_oracle(name):
    text = CASES[name]()
    assert _native_dump(text) == _oracle_dump(text)


def test_transform_matches_oracle_c2_size():
    """The 20,000-gate Tseitin workload (2,000 inputs, depth 40, 32 outputs)."""
    inst = tseitin_random_circuit(2000, 20000, 40, 32, seed=1)
    text = inst.dimacs()
    assert _native_dump(text) == _oracle_dump(text)
    c = P.Circuit.build(P.Cnf.from_dimacs(text))
    assert c.stats["n_gates"] == 20000 and c.stats["n_pi"] == 2000 and c.stats["n_outputs"] == 32
    assert c.stats["n_cone_levels"] == 40 and c.stats["max_span"] <= 4


@pytest.mark.parametrize("kind,n", [("OR", 3), ("AND", 3), ("NAND", 2), ("XOR", 3), ("XNOR", 2)])
def test_signatures_match_oracle(kind, n):
    from tests.test_oracle_pins import _sig_clauses
    text = dimacs_text(n + 1, _sig_clauses(kind, n))
    assert _native_dump(text) == _oracle_dump(text)


def test_random_cnfs_match_oracle():
    """Mixed instances: Tseitin gates with interleaved unit clauses and random clauses."""
    import numpy as np
    rng = np.random.default_rng(7)
    for trial in range(20):
        inst = tseitin_random_circuit(12, 30, 5, 2, seed=trial)
        cl = list(inst.clauses)
        for _ in range(int(rng.integers(0, 6))):
            k = int(rng.integers(1, 4))
            vs = rng.choice(inst.n_vars, k, replace=False) + 1
            cl.insert(int(rng.integers(0, len(cl) + 1)), [int(v) * int(rng.choice([-1, 1])) for v in vs])
        text = dimacs_text(inst.n_vars, cl)
        assert _native_dump(text) == _oracle_dump(text), trial


@pytest.mark.parametrize("text", ["p cnf 3 2\n1 2 0\n", "p cnf 2 1\n1 3 0\n", "1 2 0\n", "p cnf 2 1\n1 2\n",
                                  "p cnf x 1\n1 0\n", "p cnf 2 1\n1 q 0\n"])
def test_parse_errors(text):
    with pytest.raises(P.SatError) as e:
        P.Cnf.from_dimacs(text)
    assert e.value.status == -1


def test_empty_clause_is_trivially_unsat():
    cnf = P.Cnf.from_dimacs("p cnf 2 2\n1 2 0\n0\n")
    with pytest.raises(P.SatError) as e:
        P.Circuit.build(cnf)
    assert e.value.status == -6


def test_parse_counts_and_comments():
    cnf = P.Cnf.from_dimacs("c x\np cnf 3 2\n1 -2\n 3 0 -1\n0\n%\n0\n")
    assert cnf.info() == (3, 2, 4)


def test_ops_reduction_statistic():
    """Fig. 5 (middle): 2-input gate equivalents of the CNF vs the circuit."""
    c = P.Circuit.build(P.Cnf.from_dimacs(fig1_example_dimacs()))
    # CNF: 21 clauses of 2-3 literals -> sum(len-1) + 20 ANDs; circuit: 6 gates (2 MUXes), 1 output
    assert c.stats["ops_cnf"] == sum(len(x) - 1 for x in parse_dimacs(fig1_example_dimacs())[1]) + 20
    assert c.stats["ops_circuit"] == 6
