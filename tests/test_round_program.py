"""Host side of the instance-compiled round kernel: the generated program for a circuit
within the limits compiles with NVRTC for sm_103a without register spills (no GPU needed),
and a circuit beyond them is refused."""
import re

import pytest

from workloads import tseitin_random_circuit, planted_3sat, fig1_example_dimacs, dimacs_text


def _circuit(text):
    import paper_2502_08673_b300 as P
    cnf = P.Cnf.from_dimacs(text)
    return P, P.Circuit.build(cnf)


@pytest.mark.parametrize("text", [fig1_example_dimacs(), tseitin_random_circuit(50, 50, 5, 4, seed=1).dimacs(),
                                  planted_3sat(20, 60, 2).dimacs(), dimacs_text(8, [])],
                         ids=["fig1", "paper_50_50_d5", "planted3sat_20_60", "no_clauses_8"])
def test_round_program_compiles_without_spills(text):
    P, circ = _circuit(text)
    src = circ.round_program()
    assert 'extern "C" __global__' in src and "sat_round_gd_kernel" in src
    # the circuit is the code: no index loads, no shared memory, no barriers
    assert "__shared__" not in src and "__syncthreads" not in src
    st = circ.stats
    assert src.count("= sat::gate_apply(") == st["n_cone_gates"]
    assert src.count("= sat::sigmoidf_(") == st["n_cone_pi"]
    log = circ.round_program(compile=True)
    assert re.search(r"0 bytes stack frame, 0 bytes spill stores, 0 bytes spill loads", log), log
    regs = int(re.search(r"Used (\d+) registers", log).group(1))
    assert regs <= 255


def test_round_program_refuses_large_circuits():
    P, circ = _circuit(tseitin_random_circuit(64, 640, 16, 8, seed=3).dimacs())
    with pytest.raises(P.SatError, match="too many relaxed values"):
        circ.round_program()
