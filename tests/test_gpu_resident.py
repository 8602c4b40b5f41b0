"""The shared-memory resident step kernel against the tiled one and the FP64 oracle.

Both kernels perform the same operations in the same order, so V, m, v and the loss
must be bit-identical for every activation type, optimiser, per-sample Adam ages and
ragged batches; the resident kernel's trajectory is also compared with the oracle's.
"""
import numpy as np
import pytest

import oracle
from workloads import tseitin_random_circuit, planted_3sat, fig1_example_dimacs, normal_logits

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SMALL = {
    "fig1": fig1_example_dimacs,
    "planted3sat_50_200": lambda: planted_3sat(50, 200, 1).dimacs(),
    "tseitin_64_640_d16": lambda: tseitin_random_circuit(64, 640, 16, 8, seed=3).dimacs(),
    "tseitin_50_50_d5": lambda: tseitin_random_circuit(50, 50, 5, 4, seed=1).dimacs(),
}


def _plan(text):
    import paper_2502_08673_b300 as P
    cnf = P.Cnf.from_dimacs(text)
    circ = P.Circuit.build(cnf)
    return P, P.Plan.create(circ, cnf)


def _run(P, plan, kind, V0, opt, act_dtype, t0, n_steps, age=None):
    plan.set_step_kernel(kind)
    B = V0.shape[1]
    V = V0.clone()
    g = torch.Generator(device="cpu").manual_seed(1)
    m = (0.01 * torch.randn(V0.shape, generator=g)).to(V0.device)
    v = (0.001 * torch.rand(V0.shape, generator=g)).to(V0.device)
    act, adj = P.new_act(plan, B, act_dtype), P.new_adj(plan, B)
    loss = torch.full((B,), -1.0, device=V0.device)
    P.sat_steps(plan, opt, V, m, v, act, adj, t0, n_steps, loss=loss, act_dtype=act_dtype, age=age)
    torch.cuda.synchronize()
    return V, m, v, loss


@pytest.mark.parametrize("name", sorted(SMALL))
@pytest.mark.parametrize("act_dtype", ["f32", "bf16", "f16"])
def test_resident_bit_identical_to_tiled(gpu, name, act_dtype):
    P, plan = _plan(SMALL[name]())
    assert plan.step_kernel(act_dtype) == "resident"
    for B, optname, aged in ((77, "adam", False), (1000, "adam", True), (33, "gd", False), (130, "gd", True)):
        V0 = torch.tensor(normal_logits(B, plan.n_pi, seed=B).T.copy(), device=gpu)
        age = torch.randint(0, 50, (B,), dtype=torch.int32, device=gpu) if aged else None
        opt = P.opt_params(optname, lr=0.05)
        a = _run(P, plan, "tiled", V0, opt, act_dtype, 3, 9, age)
        b = _run(P, plan, "resident", V0, opt, act_dtype, 3, 9, age)
        for x, y, what in zip(a, b, ("V", "m", "v", "loss")):
            assert torch.equal(x, y), (name, act_dtype, B, optname, aged, what,
                                       (x - y).abs().max().item())
    plan.set_step_kernel("auto")


def test_resident_trajectory_vs_oracle(gpu):
    """Five GD steps (Eq. 9) on the resident kernel: GPU FP32 vs oracle FP64."""
    text = SMALL["tseitin_64_640_d16"]()
    P, plan = _plan(text)
    plan.set_step_kernel("resident")
    orc = oracle.Oracle(text)
    B = 100
    V0 = normal_logits(B, orc.n_pi, seed=2)
    V = torch.tensor(V0.T.copy(), device=gpu)
    m, v = torch.zeros_like(V), torch.zeros_like(V)
    loss = torch.empty(B, device=gpu)
    P.sat_steps(plan, P.opt_params("gd", lr=1.0), V, m, v, P.new_act(plan, B), P.new_adj(plan, B), 1, 5, loss=loss)
    trace = []
    res = oracle.sample_round(orc.flat, orc.n_vars, orc.clauses, V0.astype(np.float64), steps=5, lr=1.0, opt="gd",
                              trace=trace)
    torch.cuda.synchronize()
    np.testing.assert_allclose(V.cpu().numpy().T, res["V"], rtol=0, atol=1e-4)
    np.testing.assert_allclose(loss.cpu().numpy(), trace[-1][1], rtol=0, atol=1e-4)


def test_kernel_choice(gpu):
    """AUTO takes the resident kernel exactly when the plan's state fits its shared memory."""
    import paper_2502_08673_b300 as P
    _, small = _plan(SMALL["planted3sat_50_200"]())
    assert small.step_kernel("f32") == "resident"
    small.set_step_kernel("tiled")
    assert small.step_kernel("f32") == "tiled"
    _, big = _plan(tseitin_random_circuit(2000, 20000, 40, 32, seed=1).dimacs())
    assert big.step_kernel("f32") == "tiled" and big.step_kernel("bf16") == "tiled"
    with pytest.raises(P.SatError) as e:
        big.set_step_kernel("resident")
    assert e.value.status == -2
    assert big.step_kernel("f32") == "tiled"


def test_sampler_same_solutions_on_both_kernels(gpu):
    """sat_sample returns the same distinct set with either kernel (plain and early exit)."""
    import paper_2502_08673_b300 as P
    text = planted_3sat(50, 200, 1).dimacs()
    cnf = P.Cnf.from_dimacs(text)
    circ = P.Circuit.build(cnf)
    kw = dict(n_wanted=10 ** 9, batch=1024, steps=100, max_rounds=2, lr=0.1, seed=3)
    for extra in ({}, dict(check_every=20, max_age=60)):
        a = P.sample(circ, cnf, step_kernel="tiled", **kw, **extra)
        b = P.sample(circ, cnf, step_kernel="resident", **kw, **extra)
        assert len(a) > 0
        assert np.array_equal(a.words(), b.words())


@pytest.mark.parametrize("act_dtype", ["f32", "bf16", "f16"])
def test_resident_two_samples_per_lane_bit_identical_to_tiled(gpu, act_dtype):
    """Batches of at least 148 x 64 x 8 samples run the resident kernel with two samples per
    lane (64 per CTA, pairs through the packed FP32 fma) on narrow circuits: the same values
    as the tiled kernel, bit for bit, with a ragged last CTA, Adam with ages and GD."""
    P, plan = _plan(SMALL["tseitin_50_50_d5"]())
    assert plan.step_kernel(act_dtype) == "resident"
    B = 148 * 64 * 8 + 77
    V0 = torch.tensor(normal_logits(B, plan.n_pi, seed=4).T.copy(), device=gpu)
    for optname, aged in (("adam", True), ("gd", False)):
        age = torch.randint(0, 50, (B,), dtype=torch.int32, device=gpu) if aged else None
        opt = P.opt_params(optname, lr=0.05)
        a = _run(P, plan, "tiled", V0, opt, act_dtype, 3, 6, age)
        b = _run(P, plan, "resident", V0, opt, act_dtype, 3, 6, age)
        for x, y, what in zip(a, b, ("V", "m", "v", "loss")):
            assert torch.equal(x, y), (act_dtype, optname, what, (x - y).abs().max().item())
    plan.set_step_kernel("auto")
