"""The instance-compiled round kernel (plain GD, the paper's own setting of Section IV)
against the separate kernels it fuses, bit for bit, and against the FP64 oracle.

sat_round_gd runs init_normal, the FP32 GD steps (Eq. 5-9), the threshold, the Boolean
pass and the check of the original clauses in one launch; the keys, validity words and
final logits must equal those of the separate calls exactly (the same device functions
in the same order), for every batch size including partial warps and partial quads.
"""
import numpy as np
import pytest

import oracle
from workloads import tseitin_random_circuit, planted_3sat, fig1_example_dimacs, dimacs_text

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# circuits within the kernel's limits: the paper-setting stand-in (inputs outside the
# outputs' cone), Fig. 1 (6 inputs: a partial Philox quad), planted 3-SAT (every input in
# the cone, 254 registers), Tseitin circuits with many unconstrained gates and 100 inputs
INSTANCES = {
    "paper_50_50_d5": lambda: tseitin_random_circuit(50, 50, 5, 4, seed=1).dimacs(),
    "fig1": fig1_example_dimacs,
    "planted3sat_20_60": lambda: planted_3sat(20, 60, 2).dimacs(),
    "tseitin_40_120_d6": lambda: tseitin_random_circuit(40, 120, 6, 3, seed=5).dimacs(),
    "tseitin_100_200_d8": lambda: tseitin_random_circuit(100, 200, 8, 6, seed=7).dimacs(),
    # edge cases: outputs that are bare inputs (unit clauses; no gate in the cone), the
    # direct-CNF relaxation (every variable an input, 3-input ORs lowered to gates), a CNF
    # with no clauses (no cone at all; every sample valid)
    "units_100": lambda: dimacs_text(100, [[v if (v * 7919) % 3 else -v] for v in range(65, 101)]),
    "direct_planted3sat_20_60": lambda: planted_3sat(20, 60, 2).dimacs(),
    "no_clauses_8": lambda: dimacs_text(8, []),
}
DIRECT = {"direct_planted3sat_20_60"}


def _plan(text, direct=False):
    import paper_2502_08673_b300 as P
    cnf = P.Cnf.from_dimacs(text)
    circ = P.Circuit.build(cnf, direct=direct)
    return P, cnf, circ, P.Plan.create(circ, cnf)


def _separate(P, plan, B, lr, steps, seed, rnd, scale):
    ws = P.new_workspace(plan, B)
    P.sat_init_normal(plan, ws.V, seed=seed, round_=rnd, scale=scale)
    if steps > 0:
        P.sat_steps(plan, P.opt_params("gd", lr=lr), ws.V, ws.m, ws.v, ws.act, ws.adj, 1, steps)
    P.sat_threshold(plan, ws.V, ws.bits, ws.keys)
    P.sat_hard_eval(plan, ws.bits, B)
    P.sat_cnf_check(plan, ws.bits, ws.valid, B)
    return ws.V, ws.keys, ws.valid


def _compiled(P, plan, B, lr, steps, seed, rnd, scale, with_V=True):
    n_pi, kw = plan.info["n_pi"], max(1, plan.info["key_words"])
    keys = torch.full((B, kw), -1, dtype=torch.int32, device="cuda")
    valid = torch.full(((B + 31) // 32,), -1, dtype=torch.int32, device="cuda")
    V = torch.full((n_pi, B), float("nan"), device="cuda") if with_V else None
    P.sat_round_gd(plan, keys, valid, B, lr, steps, seed=seed, round_=rnd, scale=scale, V=V)
    return V, keys, valid


@pytest.mark.parametrize("name", sorted(INSTANCES))
def test_round_equals_separate_kernels(gpu, name):
    P, cnf, circ, plan = _plan(INSTANCES[name](), direct=name in DIRECT)
    info = plan.round_info(compile=True)
    assert info["available"] == 1 and info["compiled"] == 1 and info["spill_bytes"] == 0, info
    # compiled for as many resident blocks as its registers allow
    per_thread = (info["registers"] + 7) // 8 * 8
    assert 1 <= info["min_blocks"] <= min(65536 // (per_thread * 128), 16), info
    # scales: negative (bits of the inputs outside the cone flip with the sign), and below the
    # threshold under which the kernel forms every normal even without V
    for B, lr, steps, scale in [(1, 10.0, 5, 1.0), (37, 10.0, 5, 1.0), (1000, 10.0, 0, 1.5), (4173, 10.0, 1, 1.0),
                                (4173, 0.5, 30, 0.7), (515, 10.0, 5, -0.8), (300, 10.0, 2, 1e-20)]:
        seed, rnd = 0x9E37_79B9_7F4A + B, 3 + steps
        Vs, ks, vs = _separate(P, plan, B, lr, steps, seed, rnd, scale)
        Vc, kc, vc = _compiled(P, plan, B, lr, steps, seed, rnd, scale)
        torch.cuda.synchronize()
        assert torch.equal(Vc, Vs), (name, B, steps)
        assert torch.equal(kc, ks), (name, B, steps)
        assert torch.equal(vc, vs), (name, B, steps)
        # without V the inputs outside the cone get their bits from the signs alone
        _, kn, vn = _compiled(P, plan, B, lr, steps, seed, rnd, scale, with_V=False)
        torch.cuda.synchronize()
        assert torch.equal(kn, ks), (name, B, steps, scale)
        assert torch.equal(vn, vs), (name, B, steps, scale)
    # the step kernel the separate path uses does not matter (tiled = resident, bit for bit)
    plan.set_step_kernel("tiled")
    Vs, ks, vs = _separate(P, plan, 515, 10.0, 5, 11, 12, 1.0)
    Vc, kc, vc = _compiled(P, plan, 515, 10.0, 5, 11, 12, 1.0, with_V=False)
    torch.cuda.synchronize()
    assert torch.equal(kc, ks) and torch.equal(vc, vs)


def test_angle_signs_match_sincospi(gpu):
    """The round kernel takes the threshold bits of inputs outside every output's cone from
    the signs of the Box-Muller angle's sine and cosine read off the angle's grid index; at all
    2^24 grid points those signs equal the signs of what sincospif returns (zeros included)."""
    import ctypes as C
    from paper_2502_08673_b300 import _native as N
    bad = C.c_uint32(12345)
    N.check(N.lib().sat_diag_angle_signs(C.byref(bad), None))
    assert bad.value == 0


@pytest.mark.parametrize("name", ["paper_50_50_d5", "planted3sat_20_60", "tseitin_100_200_d8"])
def test_round_against_oracle(gpu, name):
    """From the oracle's own Philox/Box-Muller logits, five FP64 GD steps (lr 1) land within
    1e-4 of the kernel's logits; the kernel's threshold, Boolean pass and clause check of
    its own logits equal the oracle's verification of them, bit for bit."""
    text = INSTANCES[name]()
    P, cnf, circ, plan = _plan(text)
    orc = oracle.Oracle(text)
    assert list(plan.pi_vars()) == orc.circuit.pis
    B, seed, rnd = 600, 77, 5
    Vc, kc, vc = _compiled(P, plan, B, 1.0, 5, seed, rnd, 1.0)
    torch.cuda.synchronize()
    V0 = oracle.init_normal(B, orc.n_pi, seed, rnd, 1.0)
    res = oracle.sample_round(orc.flat, orc.n_vars, orc.clauses, V0, steps=5, lr=1.0, opt="gd")
    got = Vc.cpu().numpy().T.astype(np.float64)
    assert np.abs(got - res["V"]).max() <= 1e-4
    ref = oracle.verify(orc.flat, orc.n_vars, orc.clauses, got)
    assert P.valid_mask(vc, B).tolist() == ref["valid"].astype(bool).tolist()
    bits = np.unpackbits(kc.cpu().numpy().view(np.uint8), axis=1, bitorder="little")[:, : orc.n_pi]
    assert (bits == ref["pi_bits"]).all()


def test_sample_plan_uses_compiled_round(gpu):
    """sat_sample with plain GD on FP32 activations goes through the compiled round (AUTO)
    and returns the same solutions as the separate kernels (step kernel forced)."""
    import paper_2502_08673_b300 as P
    text = INSTANCES["paper_50_50_d5"]()
    cnf = P.Cnf.from_dimacs(text)
    circ = P.Circuit.build(cnf)
    kw = dict(n_wanted=10 ** 9, batch=20000, steps=5, max_rounds=2, optimizer="gd", lr=10.0, seed=4)
    a = P.sample(circ, cnf, **kw)
    b = P.sample(circ, cnf, step_kernel="resident", **kw)
    assert len(a) > 10000
    assert np.array_equal(a.words(), b.words())
    # the compiled round counts the whole round as steps time (init and verify are two
    # back-to-back events each: microseconds)
    assert a.stats["ms_init"] < 0.05 and a.stats["ms_verify"] < 0.05 and a.stats["ms_steps"] > 0.0
    assert b.stats["ms_verify"] > a.stats["ms_verify"]
    n, cl = oracle.parse_dimacs(text)
    A = a.assignments()
    assign = np.zeros((len(A), n + 1), np.uint8)
    assign[:, 1:] = A
    assert oracle.cnf_check(n, cl, assign).all()


def test_round_errors(gpu):
    import paper_2502_08673_b300 as P
    _, _, _, plan = _plan(INSTANCES["fig1"]())
    keys = torch.zeros((64, 1), dtype=torch.int32, device="cuda")
    valid = torch.zeros(2, dtype=torch.int32, device="cuda")
    with pytest.raises(P.SatError, match="SAT_ERR_ARG"):
        P.sat_round_gd(plan, keys, valid, 64, 10.0, -1)
    with pytest.raises(P.SatError, match="SAT_ERR_ARG"):
        P.sat_round_gd(plan, keys, valid, 64, float("inf"), 5)
    with pytest.raises(P.SatError, match="SAT_ERR_ARG"):
        P.sat_round_gd(plan, None, valid, 64, 10.0, 5)
    V = torch.zeros((6, 32), device="cuda")  # ldv 32 < B
    with pytest.raises(P.SatError, match="SAT_ERR_ARG"):
        P.sat_round_gd(plan, keys, valid, 64, 10.0, 5, V=V)
    # a circuit beyond the limits has no round kernel
    _, _, _, big = _plan(tseitin_random_circuit(64, 640, 16, 8, seed=3).dimacs())
    assert big.round_info()["available"] == 0
    with pytest.raises(P.SatError, match="SAT_ERR_ARG"):
        P.sat_round_gd(big, keys, valid, 64, 10.0, 5)
    # B = 0 is a no-op
    P.sat_round_gd(plan, keys, valid, 0, 10.0, 5)
