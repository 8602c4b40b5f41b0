"""Level-segment recomputation and the adjoint ring.

Recomputation is a memory schedule: the backward pass evaluates a segment's unkept
levels again with the same arithmetic in the same order, so every result (V, m, v,
loss) must equal, bit for bit, the fused steps that keep every level.  Cases: the
one-CTA and the 2-CTA cluster tiles, ragged batches, FP32 and BF16 activations, Adam
with per-sample ages and GD, segment lengths from below the edge span (everything
kept) to longer than the circuit, and outputs below the top level (kept levels in the
middle of a segment).  The adjoint ring is checked through every other backward test
(it is the only adj layout); here its size is checked against its definition.
"""
import numpy as np
import pytest

from workloads import tseitin_random_circuit, planted_3sat, normal_logits, dimacs_text
from workloads.generators import _planted_values

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _plan(text):
    """A plan on the tiled step kernel (the one with act layouts; small circuits would
    otherwise run on the shared-memory resident kernel, which keeps no act scratch)."""
    import paper_2502_08673_b300 as P
    cnf = P.Cnf.from_dimacs(text)
    circ = P.Circuit.build(cnf)
    plan = P.Plan.create(circ, cnf)
    plan.set_step_kernel("tiled")
    return P, cnf, circ, plan


def _mid_output_text(seed=4):
    """Tseitin circuit (depth 24) with extra unit clauses on gates of levels 3, 9 and 17:
    outputs in the middle of segments."""
    inst = tseitin_random_circuit(96, 24 * 40, 24, 8, seed=seed)
    vals = _planted_values(inst)
    extra = []
    for l in (3, 9, 17):
        node = inst.n_pi + (l - 1) * inst.gates_per_level + 5
        extra.append([node + 1 if vals[node] else -(node + 1)])
    return dimacs_text(inst.n_vars, inst.clauses + extra)


def _run(P, plan, B, segment, opt, act_dtype, n_steps, age=None, seed=3):
    gpu = torch.device("cuda")
    V = torch.tensor(normal_logits(plan.n_pi, B, seed=seed), device=gpu)
    m, v = torch.zeros_like(V), torch.zeros_like(V)
    act = P.new_act(plan, B, act_dtype, segment=segment)
    adj = P.new_adj(plan, B)
    loss = torch.zeros(B, device=gpu)
    P.sat_steps(plan, opt, V, m, v, act, adj, 1, n_steps, loss=loss, act_dtype=act_dtype, age=age,
                segment=segment)
    torch.cuda.synchronize()
    assert plan.status() == 0
    return V, m, v, loss


CASES = [
    ("tseitin16", lambda: tseitin_random_circuit(64, 640, 16, 8, seed=3).dimacs()),
    ("tseitin40", lambda: tseitin_random_circuit(200, 2000, 40, 16, seed=5).dimacs()),
    ("mid_outputs", _mid_output_text),
    ("planted3sat", lambda: planted_3sat(50, 200, 1).dimacs()),
]


@pytest.mark.parametrize("name,text", CASES, ids=[c[0] for c in CASES])
def test_recompute_equals_stored_f32(gpu, name, text):
    P, cnf, circ, plan = _plan(text())
    W = plan.info["max_span"]
    opt = P.opt_params("adam", lr=0.1)
    B = 203  # two tiles, the second ragged; both in 2-CTA clusters
    ref = _run(P, plan, B, 0, opt, "f32", 3)
    for k in sorted({1, W, W + 1, W + 2, 2 * W + 1, 7, 100}):
        got = _run(P, plan, B, k, opt, "f32", 3)
        for a, b in zip(got, ref):
            assert torch.equal(a, b), (name, k)


def test_recompute_rows_shrink_and_sizes(gpu):
    """Kept-level accounting: segment <= max_span keeps every level; longer segments keep
    the top max_span levels of each plus two scratch buffers; the adj ring is the input
    level plus max_span + 1 slots of the widest level."""
    P, cnf, circ, plan = _plan(tseitin_random_circuit(200, 2000, 40, 16, seed=5).dimacs())
    info = plan.info
    W, n_cone, n_cpi = info["max_span"], info["n_cone"], info["n_cone_pi"]
    full_rows, adj_rows = plan.layout_rows(0)
    assert full_rows == n_cone
    # every level of this generator has 50 gates; the cone may drop a few
    assert adj_rows < n_cone and adj_rows >= n_cpi + (W + 1) * 1
    assert W == 4 and info["n_cone_levels"] == 40
    assert plan.layout_rows(W)[0] == n_cone
    # 40 levels, W = 4.  k = 6: kept 4 x 6 + 2 (the top segment is levels 37-40) = 26
    # levels, scratch 2 x 2; k = 8: 5 x 4 kept + 2 x 4; k = 12: 3 x 4 + 4 kept + 2 x 8.
    # k = 20: 8 kept + 2 x 16 = 40 levels, no saving, so the full layout is used.
    gate_rows = n_cone - n_cpi  # about 50 per level (the cone drops a few gates)
    for k, levels in ((6, 30), (8, 28), (12, 32)):
        r = plan.layout_rows(k)[0] - n_cpi
        assert abs(r - gate_rows * levels / 40) <= 0.1 * gate_rows * levels / 40, (k, r)
    assert plan.layout_rows(20)[0] == n_cone and plan.layout_rows(100)[0] == n_cone
    assert plan.scratch_elems(128) == n_cone * 128


@pytest.mark.parametrize("act_dtype", ["f32", "bf16", "f16"])
def test_recompute_full_waves_and_split_tail(gpu, act_dtype):
    """149 tiles: one full wave of one-CTA tiles plus a split tail; Adam with ages and GD."""
    P, cnf, circ, plan = _plan(tseitin_random_circuit(64, 640, 16, 8, seed=7).dimacs())
    B = 148 * 128 + 77
    rng = np.random.default_rng(2)
    age = torch.tensor(rng.choice([0, 3, 50], size=B).astype(np.int32), device=gpu)
    for opt, a in ((P.opt_params("adam", lr=0.05), age), (P.opt_params("gd", lr=0.5), None)):
        ref = _run(P, plan, B, 0, opt, act_dtype, 2, age=a, seed=11)
        got = _run(P, plan, B, 6, opt, act_dtype, 2, age=a, seed=11)
        for x, y in zip(got, ref):
            assert torch.equal(x, y)


def test_sampler_with_recompute_same_solutions(gpu):
    """sat_sample with recompute_segment returns the same distinct set as without."""
    import paper_2502_08673_b300 as P
    text = tseitin_random_circuit(64, 640, 16, 8, seed=3).dimacs()
    cnf = P.Cnf.from_dimacs(text)
    circ = P.Circuit.build(cnf)
    kw = dict(n_wanted=10 ** 9, batch=512, steps=60, max_rounds=2, lr=0.1, seed=9, step_kernel="tiled")
    a = P.sample(circ, cnf, **kw)
    b = P.sample(circ, cnf, recompute_segment=6, **kw)
    assert len(a) > 0
    assert np.array_equal(a.words(), b.words())
    c = P.sample(circ, cnf, recompute_segment=6, check_every=20, max_age=40, **kw)
    d = P.sample(circ, cnf, check_every=20, max_age=40, **kw)
    assert np.array_equal(c.words(), d.words())


@pytest.mark.parametrize("name", ["tseitin16", "mid_outputs"])
@pytest.mark.parametrize("opt_name,lr,atol", [("gd", 0.5, 2e-5), ("adam", 0.02, 1e-3)])
def test_recompute_trajectory_vs_oracle(gpu, name, opt_name, lr, atol):
    """100 recomputed steps (segments of 2 to 6 levels) against the FP64 oracle's trajectory
    from the same V0, with the bounds of the stored-layout trajectory test on the 16-level
    circuit (10x its measured FP32 drift: 1.7e-6 GD, 1.0e-4 Adam); thresholded bits agree
    wherever the oracle's logit is not within 10 x atol of 0."""
    import oracle
    text = dict(CASES)[name]()
    P, cnf, circ, plan = _plan(text)
    orc = oracle.Oracle(text)
    assert list(plan.pi_vars()) == orc.circuit.pis
    B, steps = 96, 100
    V0 = normal_logits(B, orc.n_pi, seed=8, scale=0.5)
    f32 = lambda x: float(np.float32(x))  # noqa: E731  (the GPU's FP32 constants)
    res = oracle.sample_round(orc.flat, orc.n_vars, orc.clauses, V0.astype(np.float64), steps=steps, lr=f32(lr),
                              opt=opt_name, betas=(f32(0.9), f32(0.999)), eps=f32(1e-8))
    near = np.abs(res["V"]) <= 10 * atol
    for k in (2, 5, 6):
        V = torch.tensor(V0.T.copy(), device=gpu)
        m, v = torch.zeros_like(V), torch.zeros_like(V)
        P.sat_steps(plan, P.opt_params(opt_name, lr=lr), V, m, v, P.new_act(plan, B, segment=k),
                    P.new_adj(plan, B), 1, steps, segment=k)
        torch.cuda.synchronize()
        assert plan.status() == 0
        got = V.cpu().numpy().T.astype(np.float64)
        err = np.abs(got - res["V"])
        print(f"{name} {opt_name} segment {k}: max |V - V*| after {steps} steps = {err.max():.2e}")
        assert err.max() <= atol, (k, err.max())
        assert ((got > 0) == (res["V"] > 0))[~near].all()
