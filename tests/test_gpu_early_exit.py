"""Early exit: per-sample Adam steps, retire/restart, and the sampler built on them.

The aged fused steps must equal, bit for bit, plain fused steps run separately on
each group of samples that share an age (samples are independent and the Adam
correction of a sample depends only on its own step count).  Retirement and
restarts are integer / copy work: exact.  The sampler's output is checked with
the oracle's CNF evaluation.
"""
import numpy as np
import pytest

import oracle
from workloads import tseitin_random_circuit, planted_3sat, normal_logits

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _setup(text):
    import paper_2502_08673_b300 as P
    cnf = P.Cnf.from_dimacs(text)
    circ = P.Circuit.build(cnf)
    plan = P.Plan.create(circ, cnf)
    return P, cnf, circ, plan


def test_aged_steps_equal_grouped_plain_steps(gpu):
    P, cnf, circ, plan = _setup(tseitin_random_circuit(64, 640, 16, 8, seed=3).dimacs())
    B, n_steps = 203, 3
    rng = np.random.default_rng(7)
    ages = rng.choice([0, 4, 37, 500], size=B).astype(np.int32)
    V0 = normal_logits(B, plan.n_pi, seed=9).T.copy()
    m0 = (rng.normal(size=V0.shape) * 0.1).astype(np.float32)
    v0 = (rng.random(size=V0.shape) * 0.01).astype(np.float32)
    opt = P.opt_params("adam", lr=0.05)
    V, m, v = (torch.tensor(x, device=gpu) for x in (V0, m0, v0))
    age = torch.tensor(ages, device=gpu)
    P.sat_steps(plan, opt, V, m, v, P.new_act(plan, B), P.new_adj(plan, B), 1, n_steps, age=age)
    torch.cuda.synchronize()
    assert torch.equal(age.cpu(), torch.tensor(ages))  # read only
    for a in np.unique(ages):
        cols = np.flatnonzero(ages == a)
        n = len(cols)
        Vg, mg, vg = (torch.tensor(np.ascontiguousarray(x[:, cols]), device=gpu) for x in (V0, m0, v0))
        P.sat_steps(plan, opt, Vg, mg, vg, P.new_act(plan, n), P.new_adj(plan, n), int(a) + 1, n_steps)
        torch.cuda.synchronize()
        idx = torch.tensor(cols, device=gpu)
        assert torch.equal(V[:, idx], Vg), a
        assert torch.equal(m[:, idx], mg) and torch.equal(v[:, idx], vg), a


def test_adam_bias_correction_large_t(gpu):
    """FP32 bias corrections stay within 1e-6 relative of the FP64 oracle at any t."""
    P, cnf, circ, plan = _setup(tseitin_random_circuit(64, 640, 16, 8, seed=3).dimacs())
    B = 64
    rng = np.random.default_rng(1)
    cone, _, _ = plan.var_nodes()
    cone_rows = np.array([cone[v] >= 0 for v in plan.pi_vars()])
    g = (rng.normal(size=(plan.n_pi, B)) * cone_rows[:, None]).astype(np.float32)
    for t in (1, 2, 10, 1000, 100000):
        V0 = rng.normal(size=(plan.n_pi, B)).astype(np.float32)
        m0 = (rng.normal(size=(plan.n_pi, B)) * 0.1).astype(np.float32)
        v0 = (rng.random(size=(plan.n_pi, B)) * 0.01 + 1e-4).astype(np.float32)
        Vd, md, vd = (torch.tensor(x, device=gpu) for x in (V0, m0, v0))
        P.sat_opt_update(plan, P.opt_params("adam", lr=0.1), Vd, md, vd, torch.tensor(g, device=gpu), t)
        torch.cuda.synchronize()
        Vr, mr, vr = V0.astype(np.float64), m0.astype(np.float64), v0.astype(np.float64)
        oracle.adam_step(Vr, mr, vr, g.astype(np.float64), t, 0.1, b1=float(np.float32(0.9)),
                         b2=float(np.float32(0.999)), eps=float(np.float32(1e-8)))
        # only cone rows are optimised (the others carry state here but no gradient)
        step = np.abs(Vr - V0.astype(np.float64))[cone_rows]
        err = np.abs(Vd.cpu().numpy().astype(np.float64) - Vr)[cone_rows]
        assert (err <= 1e-6 * step + 2e-7 * np.abs(Vr[cone_rows]) + 1e-7).all(), (t, float(err.max()))
        assert torch.equal(Vd.cpu()[~torch.tensor(cone_rows)], torch.tensor(V0)[~torch.tensor(cone_rows)])


def test_retire_and_restart_exact(gpu):
    P, cnf, circ, plan = _setup(planted_3sat(50, 200, 1).dimacs())
    B, k, max_age = 301, 10, 40
    W = (B + 31) // 32
    rng = np.random.default_rng(3)
    valid_bits = rng.random(B) < 0.3
    ages = rng.integers(0, 45, size=B).astype(np.int32)
    valid = torch.tensor(np.frombuffer(np.packbits(np.concatenate([valid_bits, np.zeros(W * 32 - B, bool)]),
                                                   bitorder="little").tobytes(), np.int32).copy(), device=gpu)
    age = torch.tensor(ages, device=gpu)
    restart = torch.full((W,), -1, dtype=torch.int32, device=gpu)
    P.sat_retire(valid, age, restart, k, max_age, B)
    torch.cuda.synchronize()
    want = valid_bits | (ages + k >= max_age)
    got = np.unpackbits(restart.cpu().numpy().view(np.uint8), bitorder="little")[:B].astype(bool)
    assert (got == want).all()
    assert (age.cpu().numpy() == np.where(want, 0, ages + k)).all()
    # restart from the init stream of round 7, then from a source matrix
    V0 = rng.normal(size=(plan.n_pi, B)).astype(np.float32)
    V, m, v = torch.tensor(V0, device=gpu), torch.ones(plan.n_pi, B, device=gpu), torch.ones(plan.n_pi, B, device=gpu)
    P.sat_restart(plan, restart, 5, 7, V, m, v, scale=0.5)
    ref = torch.empty(plan.n_pi, B, device=gpu)
    P.sat_init_normal(plan, ref, 5, 7, 0.5)
    torch.cuda.synchronize()
    w = torch.tensor(want, device=gpu)
    assert torch.equal(V[:, w], ref[:, w]) and torch.equal(V[:, ~w], torch.tensor(V0, device=gpu)[:, ~w])
    assert (m[:, w] == 0).all() and (v[:, w] == 0).all() and (m[:, ~w] == 1).all() and (v[:, ~w] == 1).all()
    src = torch.randn(plan.n_pi, B + 5, device=gpu)
    P.sat_restart(plan, restart, 5, 8, V, m, v, src=src[:, :B])
    torch.cuda.synchronize()
    assert torch.equal(V[:, w], src[:, :B][:, w])


def test_early_exit_sampler_planted3sat(gpu):
    """sat_sample with early exit: every solution passes the oracle's CNF check, and
    harvesting every 10 steps finds more distinct solutions than fixed rounds with
    the same descent budget."""
    import paper_2502_08673_b300 as P
    text = planted_3sat(50, 200, 1).dimacs()
    cnf = P.Cnf.from_dimacs(text)
    circ = P.Circuit.build(cnf)
    kw = dict(n_wanted=10 ** 9, batch=1024, steps=200, max_rounds=2, lr=0.1, seed=0)
    plain = P.sample(circ, cnf, **kw)
    ee = P.sample(circ, cnf, check_every=10, max_age=100, **kw)
    A = ee.assignments()
    n, cl = oracle.parse_dimacs(text)
    assign = np.zeros((len(A), n + 1), np.uint8)
    assign[:, 1:] = A
    assert len(A) == ee.stats["unique"] > 0
    assert oracle.cnf_check(n, cl, assign).all()
    assert len({a.tobytes() for a in A}) == len(A)
    assert ee.stats["rounds"] == 40  # epochs of 10 steps over the 400-step budget
    print(f"unique: fixed rounds {len(plain)}, early exit {len(A)} ({ee.stats['valid']} valid harvests, "
          f"{ee.stats['samples']} starts)")
    assert len(A) > len(plain)


def test_run_epochs_matches_c_loop(gpu):
    """The Python orchestration (run_epochs) and sat_sample's early-exit loop run the
    same kernels on the same Philox streams: identical distinct sets."""
    import paper_2502_08673_b300 as P
    text = planted_3sat(50, 200, 2).dimacs()
    cnf = P.Cnf.from_dimacs(text)
    circ = P.Circuit.build(cnf)
    plan = P.Plan.create(circ, cnf)
    B, steps, k, max_age = 512, 120, 15, 60
    ws = P.new_workspace(plan, B)
    dd = P.Dedup.create(plan, max_keys=B * (steps // k + 1), max_batch=B)
    P.run_epochs(plan, ws, P.opt_params("adam", lr=0.1), steps, k, max_age, seed=4, round_=0, dedup=dd)
    mine = {r.tobytes() for r in dd.keys()}
    sols = P.sample(circ, cnf, n_wanted=10 ** 9, batch=B, steps=steps, max_rounds=1, lr=0.1, seed=4,
                    check_every=k, max_age=max_age)
    kwords = plan.info["key_words"]
    theirs = set()
    for wrow in sols.words():
        bits = np.zeros(plan.n_vars + 1, np.uint8)
        for j in range(plan.n_vars):
            bits[j + 1] = (int(wrow[j // 64]) >> (j % 64)) & 1
        key = np.zeros(kwords, np.uint32)
        for i, var in enumerate(plan.pi_vars()):
            if bits[var]:
                key[i // 32] |= np.uint32(1) << np.uint32(i % 32)
        theirs.add(key.view(np.int32).tobytes())
    assert mine == theirs and len(mine) > 0


def test_early_exit_with_proposal_restarts(gpu):
    """sat_sample with early exit and a proposal network: restarted slots start from the
    proposal's logits (its noise of the restart round); every returned assignment is valid."""
    import paper_2502_08673_b300 as P
    text = planted_3sat(50, 200, 3).dimacs()
    cnf = P.Cnf.from_dimacs(text)
    circ = P.Circuit.build(cnf)
    plan = P.Plan.create(circ, cnf)
    B = 512
    mlp = P.Mlp.create(64, 256, plan.n_pi, max_rows=B, seed=1)
    sols = P.sample(circ, cnf, n_wanted=10 ** 9, batch=B, steps=60, max_rounds=1, lr=0.1, seed=3,
                    proposal=mlp, tau=1.0, check_every=10, max_age=30)
    A = sols.assignments()
    n, cl = oracle.parse_dimacs(text)
    assign = np.zeros((len(A), n + 1), np.uint8)
    assign[:, 1:] = A
    assert oracle.cnf_check(n, cl, assign).all()
    assert sols.stats["rounds"] == 6 and sols.stats["samples"] >= B
    # the Python orchestration on the same streams restarts from the proposal: after one epoch
    # with every sample forced to restart (max_age 1), V equals the proposal of round 1
    ws = P.new_workspace(plan, B)
    dd = P.Dedup.create(plan, max_keys=4 * B, max_batch=B)
    P.run_epochs(plan, ws, P.opt_params("adam", lr=0.1), 1, 1, 1, seed=3, round_=0, dedup=dd, proposal=mlp)
    expect = torch.empty_like(ws.V)
    mlp.propose(expect, 3, 1, 1.0)
    torch.cuda.synchronize()
    assert torch.equal(ws.V, expect)
    assert (ws.m == 0).all() and (ws.v == 0).all() and (ws.age == 0).all()
