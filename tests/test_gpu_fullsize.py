"""Parity at the full size of the benchmarked workload, in the launch configuration it is timed in.

Tseitin random circuit, 2,000 inputs, 20,000 gates, depth 40, 32 outputs, batch 65,536: 512 tiles,
of which 444 run as one CTA each (three full waves on 148 SMs) and 68 as 2-CTA clusters.  Checked
on samples drawn from both kinds of tile against the FP64 oracle (GD trajectory and loss), bit for
bit against the unfused kernels (BF16, 24-warp CTAs), and through the verification stages
(validity bit-exact on the samples, the distinct count against the keys of the whole batch).
"""
import numpy as np
import pytest

import oracle
from workloads import tseitin_random_circuit, normal_logits

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

B = 65536


@pytest.fixture(scope="module")
def setup():
    import paper_2502_08673_b300 as P
    inst = tseitin_random_circuit(2000, 20000, 40, 32, seed=1)
    text = inst.dimacs()
    cnf = P.Cnf.from_dimacs(text)
    plan = P.Plan.create(P.Circuit.build(cnf), cnf)
    orc = oracle.Oracle(text)
    assert list(plan.pi_vars()) == orc.circuit.pis
    return P, inst, plan, orc


def _samples(seed=0):
    """Samples in the first and last one-CTA tiles (0, 443), the first and last split tiles
    (444, 511), lane boundaries inside them, and a few random ones."""
    idx = [t * 128 + o for t in (0, 1, 443, 444, 445, 511) for o in (0, 3, 4, 77, 127)]
    idx += list(np.random.default_rng(seed).integers(0, B, 10))
    return np.array(sorted(set(idx)))


def test_fullsize_gd_trajectory_and_loss(gpu, setup):
    P, inst, plan, orc = setup
    V0 = normal_logits(B, orc.n_pi, seed=21)
    V = torch.tensor(V0.T.copy(), device=gpu)
    m, v = torch.zeros_like(V), torch.zeros_like(V)
    act, adj = P.new_act(plan, B), P.new_adj(plan, B)
    loss = torch.empty(B, device=gpu)
    P.sat_steps(plan, P.opt_params("gd", lr=0.5), V, m, v, act, adj, 1, 3, loss=loss)
    torch.cuda.synchronize()
    assert plan.status() == 0
    idx = _samples()
    trace = []
    res = oracle.sample_round(orc.flat, orc.n_vars, orc.clauses, V0[idx].astype(np.float64), steps=3, lr=0.5,
                              opt="gd", trace=trace)
    got = V[:, torch.tensor(idx, device=gpu)].cpu().numpy().T
    np.testing.assert_allclose(got, res["V"], rtol=0, atol=1e-4)
    np.testing.assert_allclose(loss.cpu().numpy()[idx], trace[-1][1], rtol=0, atol=1e-4)
    assert torch.isfinite(V).all() and torch.isfinite(loss).all()


def test_fullsize_bf16_fused_equals_unfused(gpu, setup):
    """Fused steps (444 one-CTA tiles + 68 split tiles, 24-warp CTAs) = forward, backward,
    update launched separately (one CTA per tile), bit for bit, with BF16 activations."""
    P, inst, plan, orc = setup
    V0 = torch.tensor(normal_logits(B, orc.n_pi, seed=5).T.copy(), device=gpu)
    opt = P.opt_params("adam", lr=0.1)
    act, adj = P.new_act(plan, B, "bf16"), P.new_adj(plan, B)
    Va, ma, va = V0.clone(), torch.zeros_like(V0), torch.zeros_like(V0)
    P.sat_steps(plan, opt, Va, ma, va, act, adj, 1, 2, act_dtype="bf16")
    Vb, mb, vb = V0.clone(), torch.zeros_like(V0), torch.zeros_like(V0)
    gV = torch.zeros_like(V0)
    for t in (1, 2):
        P.sat_forward(plan, Vb, act, act_dtype="bf16")
        P.sat_backward(plan, Vb, act, adj, gV, act_dtype="bf16")
        P.sat_opt_update(plan, opt, Vb, mb, vb, gV, t)
    torch.cuda.synchronize()
    assert plan.status() == 0
    assert torch.equal(Va, Vb) and torch.equal(ma, mb) and torch.equal(va, vb)


def test_fullsize_verification_and_dedup(gpu, setup):
    """Near-planted logits (0.1 % of inputs flipped, a quarter of the rows duplicated): validity on
    the samples equals the oracle's; the distinct count equals the distinct valid keys of the batch."""
    P, inst, plan, orc = setup
    rng = np.random.default_rng(9)
    base = np.where(inst.planted == 1, 1.0, -1.0).astype(np.float32)
    V = np.tile(base, (B, 1))
    V[rng.random(V.shape) < 0.001] *= -1
    V[rng.integers(0, B, B // 4)] = V[rng.integers(0, B, B // 4)]
    ws = P.new_workspace(plan, B)
    ws.V.copy_(torch.tensor(V.T.copy()))
    dd = P.Dedup.create(plan, max_keys=B, max_batch=B)
    P.sat_threshold(plan, ws.V, ws.bits, ws.keys)
    P.sat_hard_eval(plan, ws.bits, B)
    P.sat_cnf_check(plan, ws.bits, ws.valid, B)
    dd.insert(ws.keys, ws.valid, B)
    torch.cuda.synchronize()
    valid = P.valid_mask(ws.valid, B)
    idx = _samples(1)
    ref = oracle.verify(orc.flat, orc.n_vars, orc.clauses, V[idx])
    assert valid[idx].tolist() == ref["valid"].astype(bool).tolist()
    assert 0 < valid.sum() < B
    keys = ws.keys.cpu().numpy()
    assert dd.count() == len(np.unique(keys[valid], axis=0))


def test_fullsize_sample_every_returned_assignment_passes_oracle(gpu, setup):
    """sat_sample at the benchmarked configuration (batch 65,536, 500 Adam steps, lr 0.1, FP32,
    one round, from host CNF and circuit objects): every returned full assignment satisfies every
    original clause by the oracle's CNF check, the assignments are pairwise distinct, and each one
    is the Boolean completion of its own primary-input bits by the oracle's circuit (the
    threshold, keep-satisfiable, keep-non-redundant step at the end of Section III-A)."""
    P, inst, plan, orc = setup
    cnf = P.Cnf.from_dimacs(inst.dimacs())
    circ = P.Circuit.build(cnf)
    sols = P.sample(circ, cnf, n_wanted=10 ** 12, batch=B, steps=500, max_rounds=1, lr=0.1, seed=0)
    n = len(sols)
    # the workload's measured valid fraction is about one half; require a substantial set
    assert n > B // 4, n
    words = sols.words()
    assert np.unique(words, axis=0).shape[0] == n
    pis = np.array(orc.circuit.pis) - 1
    checked = 0
    for lo in range(0, n, 4096):
        w = words[lo:lo + 4096]
        bits = np.unpackbits(w.view(np.uint8), axis=1, bitorder="little")[:, : orc.n_vars]
        assign = np.zeros((bits.shape[0], orc.n_vars + 1), np.uint8)
        assign[:, 1:] = bits
        ok = oracle.cnf_check(orc.n_vars, orc.clauses, assign)
        assert ok.all(), np.nonzero(ok == 0)[0][:10] + lo
        completed = oracle.full_assignment(orc.flat, oracle.hard_eval(orc.flat, bits[:, pis]))
        assert np.array_equal(completed, assign)
        checked += bits.shape[0]
    assert checked == n


def test_fullsize_chosen_form_every_returned_assignment_passes_oracle(gpu, setup):
    """sat_sample in the chosen form's configuration (BF16 activations, initial logits from the
    proposal network with tau = 2, 120 Adam steps at lr 0.3, early exit every 40 steps with
    restarts after 160; batch 65,536): every returned assignment satisfies every original clause
    by the oracle's CNF check, is distinct, and is the Boolean completion of its own input bits.
    The network keeps its seeded initial weights: what is checked is that lower-precision storage
    and proposed starts never let an invalid assignment through."""
    P, inst, plan, orc = setup
    cnf = P.Cnf.from_dimacs(inst.dimacs())
    circ = P.Circuit.build(cnf)
    mlp = P.Mlp.create(64, 256, plan.info["n_pi"], max_rows=B, seed=3)
    sols = P.sample(circ, cnf, n_wanted=10 ** 12, batch=B, steps=120, max_rounds=1, lr=0.3, seed=1,
                    act_dtype="bf16", proposal=mlp, tau=2.0, check_every=40, max_age=160)
    n = len(sols)
    assert n > 1000, n
    words = sols.words()
    assert np.unique(words, axis=0).shape[0] == n
    pis = np.array(orc.circuit.pis) - 1
    for lo in range(0, n, 4096):
        w = words[lo:lo + 4096]
        bits = np.unpackbits(w.view(np.uint8), axis=1, bitorder="little")[:, : orc.n_vars]
        assign = np.zeros((bits.shape[0], orc.n_vars + 1), np.uint8)
        assign[:, 1:] = bits
        ok = oracle.cnf_check(orc.n_vars, orc.clauses, assign)
        assert ok.all(), np.nonzero(ok == 0)[0][:10] + lo
        completed = oracle.full_assignment(orc.flat, oracle.hard_eval(orc.flat, bits[:, pis]))
        assert np.array_equal(completed, assign)
    print(f"chosen-form configuration: {n} distinct assignments, all valid")
