"""Parity at the full sizes of the deep workloads, in the launch shapes they are timed in.

* 80,000-gate Tseitin circuit (5,000 inputs, depth 80, 32 outputs), batch 262,144: 2,048 tiles,
  every one a one-CTA tile (13 full waves of 148 and a last wave of 124, too large to split).
* 1,000,000-gate Tseitin circuit (50,000 inputs, depth 200, 256 outputs), batch 8,192: 64 tiles,
  every one a 2-CTA cluster (the split mode of a partial wave), BF16 activations with level-segment
  recomputation every 16 levels.

The oracle cannot run these batches, so it checks sampled samples one by one (tiles at both ends,
lane boundaries, random ones): initial logits come from the device's Philox stream and are handed
to the FP64 oracle exactly (FP32 values are exact in FP64).  One fused GD step with lr = 2^20 (a
power of two, so lr * g is exact inside the update's fma) leaves V1 = fl(V0 - lr g), so
(V0 - V1) / lr is the kernel's gradient up to half an ulp of V1 divided by lr; it is held to the
gradient bound of the small-size parity tests (1e-4 of the sum of absolute chain-rule terms plus
1e-7 of the sample's largest such sum).  With BF16 storage the per-step error against FP64 is
stated (printed) and held to a regression bound; the BF16 kernels are checked bit for bit against
another schedule of the same arithmetic (unfused kernels, the stored-activation layout).
Verification (threshold, Boolean pass, CNF check, dedup) is checked on near-planted logits.
"""
import numpy as np
import pytest

import oracle
from workloads import tseitin_random_circuit

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SHAPES = {
    # name: (inputs, gates, depth, outputs, batch)
    "tseitin80k": (5000, 80000, 80, 32, 262144),
    "tseitin1m": (50000, 1000000, 200, 256, 8192),
}


def _build(name):
    import paper_2502_08673_b300 as P
    n_pi, n_gates, depth, n_out, B = SHAPES[name]
    inst = tseitin_random_circuit(n_pi, n_gates, depth, n_out, seed=1)
    text = inst.dimacs()
    cnf = P.Cnf.from_dimacs(text)
    plan = P.Plan.create(P.Circuit.build(cnf), cnf)
    orc = oracle.Oracle(text)
    assert list(plan.pi_vars()) == orc.circuit.pis
    return P, inst, plan, orc, B


@pytest.fixture(scope="module")
def c80k():
    return _build("tseitin80k")


@pytest.fixture(scope="module")
def c1m():
    return _build("tseitin1m")


def _samples(B, seed):
    """First, second and last tiles at lane boundaries, and random samples."""
    tiles = B // 128
    idx = [t * 128 + o for t in (0, 1, tiles // 2, tiles - 1) for o in (0, 3, 4, 64, 127)]
    idx += list(np.random.default_rng(seed).integers(0, B, 8))
    return np.array(sorted(set(idx)))


LR = 2.0 ** 20


def _one_gd_step(P, plan, B, act_dtype, segment=0, seed=3):
    """V0 from Philox, one fused GD step with lr = LR; returns V0, V1 and the loss at V0."""
    n_pi = plan.info["n_pi"]
    V = torch.empty((n_pi, B), dtype=torch.float32, device="cuda")
    P.sat_init_normal(plan, V, seed, 0)
    V0 = V.clone()
    loss = torch.empty(B, device="cuda")
    # GD keeps no optimiser state (m, v NULL)
    P.sat_steps(plan, P.opt_params("gd", lr=LR), V, None, None, P.new_act(plan, B, act_dtype, segment=segment),
                P.new_adj(plan, B), 1, 1, loss=loss, act_dtype=act_dtype, segment=segment)
    torch.cuda.synchronize()
    assert plan.status() == 0
    return V0, V, loss


def _oracle_at(orc, V0, V1, loss, idx):
    """Kernel gradient, oracle gradient and its magnitude, losses at the sampled samples."""
    cols = torch.tensor(idx, device=V0.device)
    v0 = V0[:, cols].cpu().numpy().T.astype(np.float64)
    v1 = V1[:, cols].cpu().numpy().T.astype(np.float64)
    vals, loss_ref = oracle.forward(orc.flat, v0)
    gref, _ = oracle.backward(orc.flat, vals)
    gmag = oracle.backward_magnitude(orc.flat, vals)
    return (v0 - v1) / LR, v1, gref, gmag, loss.cpu().numpy()[idx].astype(np.float64), loss_ref


def _check_fp32(orc, V0, V1, loss, idx, n_out):
    g, v1, gref, gmag, lg, lref = _oracle_at(orc, V0, V1, loss, idx)
    tol = 1e-4 * gmag + 1e-7 * gmag.max(axis=1, keepdims=True) + 2.0 ** -24 * np.abs(v1) / LR + 1e-30
    ratio = np.abs(g - gref) / tol
    print(f"FP32: max |g - g*| / bound = {ratio.max():.3g}, max |loss - loss*| = {np.abs(lg - lref).max():.3g}")
    assert (ratio <= 1).all(), (np.argwhere(ratio > 1)[:5], ratio.max())
    np.testing.assert_allclose(lg, lref, rtol=0, atol=1e-5 * n_out)
    assert np.abs(gref).max() > 0


# Regression bounds on the stated per-step error of 16-bit activation storage (loss max
# relative, dL/dV over the sum of absolute terms): a few times the largest value measured on
# the 20k-, 80k- and 1M-gate workloads (BF16 0.4 % and 0.21; FP16 0.05 % and 0.08).
BOUNDS = {"bf16": (1e-2, 0.5), "f16": (2e-3, 0.25)}


def _bf16_error(orc, V0, V1, loss, idx):
    """Per-step error of BF16 activation storage against FP64: loss (max relative) and dL/dV
    (max |g - g*| over the sum of absolute chain-rule terms plus 1e-3 of the sample's largest)."""
    g, _, gref, gmag, lg, lref = _oracle_at(orc, V0, V1, loss, idx)
    loss_rel = float((np.abs(lg - lref) / np.maximum(np.abs(lref), 1e-30)).max())
    g_err = float((np.abs(g - gref) / (gmag + 1e-3 * gmag.max(axis=1, keepdims=True) + 1e-30)).max())
    return loss_rel, g_err


def test_80k_fp32_gradient_and_loss(gpu, c80k):
    P, inst, plan, orc, B = c80k
    V0, V1, loss = _one_gd_step(P, plan, B, "f32")
    _check_fp32(orc, V0, V1, loss, _samples(B, 0), plan.n_outputs)
    assert torch.isfinite(V1).all() and torch.isfinite(loss).all()


def test_80k_bf16_fused_equals_unfused_and_error(gpu, c80k):
    """2 fused Adam steps with BF16 activations = forward, backward, update launched separately,
    bit for bit; then one fused GD step's error against FP64 on the sampled samples."""
    P, inst, plan, orc, B = c80k
    opt = P.opt_params("adam", lr=0.1)
    n_pi = plan.info["n_pi"]
    V0 = torch.empty((n_pi, B), dtype=torch.float32, device=gpu)
    P.sat_init_normal(plan, V0, 5, 0)
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
    del act, adj, Va, ma, va, Vb, mb, vb, gV, V0
    torch.cuda.empty_cache()
    for dtype in ("bf16", "f16"):
        V0, V1, loss = _one_gd_step(P, plan, B, dtype)
        loss_rel, g_err = _bf16_error(orc, V0, V1, loss, _samples(B, 1))
        print(f"80k gates, {dtype} activations: loss max rel {loss_rel:.3g}, dL/dV err / sum|terms| {g_err:.3g}")
        assert loss_rel <= BOUNDS[dtype][0] and g_err <= BOUNDS[dtype][1]


def _near_planted(inst, B, n_pi, flip, seed, device):
    """Logits +-1 at the planted input with a fraction `flip` of entries negated and a quarter
    of the rows duplicated, built on the device; returns V [n_pi][B]."""
    g = torch.Generator(device=device).manual_seed(seed)
    base = torch.tensor(np.where(inst.planted == 1, 1.0, -1.0).astype(np.float32), device=device)
    V = base[:, None].expand(n_pi, B).clone()
    V[torch.rand((n_pi, B), generator=g, device=device) < flip] *= -1
    src = torch.randint(0, B, (B // 4,), generator=g, device=device)
    dst = torch.randint(0, B, (B // 4,), generator=g, device=device)
    V[:, dst] = V[:, src]
    return V


def _check_verification(P, inst, plan, orc, B, flip, seed):
    n_pi = plan.info["n_pi"]
    V = _near_planted(inst, B, n_pi, flip, seed, "cuda")
    W = (B + 31) // 32
    bits = torch.zeros((plan.info["n_nodes"], W), dtype=torch.int32, device="cuda")
    keys = torch.zeros((B, max(1, plan.info["key_words"])), dtype=torch.int32, device="cuda")
    valid = torch.zeros(W, dtype=torch.int32, device="cuda")
    dd = P.Dedup.create(plan, max_keys=B, max_batch=B)
    P.sat_threshold(plan, V, bits, keys)
    P.sat_hard_eval(plan, bits, B)
    P.sat_cnf_check(plan, bits, valid, B)
    dd.insert(keys, valid, B)
    torch.cuda.synchronize()
    ok = P.valid_mask(valid, B)
    idx = _samples(B, seed)
    ref = oracle.verify(orc.flat, orc.n_vars, orc.clauses, V[:, torch.tensor(idx, device="cuda")].cpu().numpy().T)
    assert ok[idx].tolist() == ref["valid"].astype(bool).tolist()
    assert 0 < ok.sum() < B
    k = keys.cpu().numpy()
    assert dd.count() == len(np.unique(k[ok], axis=0))
    print(f"valid {int(ok.sum())} of {B}, distinct {dd.count()}")


def test_80k_verification_and_dedup(gpu, c80k):
    P, inst, plan, orc, B = c80k
    _check_verification(P, inst, plan, orc, B, 2e-4, 7)


def test_1m_fp32_gradient_and_loss(gpu, c1m):
    P, inst, plan, orc, B = c1m
    V0, V1, loss = _one_gd_step(P, plan, B, "f32")
    _check_fp32(orc, V0, V1, loss, _samples(B, 2), plan.n_outputs)


def test_1m_bf16_recompute_equals_stored_and_error(gpu, c1m):
    """The timed form of this workload (BF16 activations, recomputation every 16 levels): 2 fused
    Adam steps equal the stored-activation layout's bit for bit; one GD step's error against FP64."""
    P, inst, plan, orc, B = c1m
    opt = P.opt_params("adam", lr=0.1)
    n_pi = plan.info["n_pi"]
    V0 = torch.empty((n_pi, B), dtype=torch.float32, device=gpu)
    P.sat_init_normal(plan, V0, 9, 0)
    out = []
    for seg in (0, 16):
        V, m, v = V0.clone(), torch.zeros_like(V0), torch.zeros_like(V0)
        loss = torch.empty(B, device=gpu)
        act = P.new_act(plan, B, "bf16", segment=seg)
        P.sat_steps(plan, opt, V, m, v, act, P.new_adj(plan, B), 1, 2, loss=loss, act_dtype="bf16", segment=seg)
        torch.cuda.synchronize()
        assert plan.status() == 0
        out.append((V, m, v, loss))
        del act
    assert plan.layout_rows(16)[0] < plan.info["n_cone"]
    for x, y in zip(*out):
        assert torch.equal(x, y)
    del out
    torch.cuda.empty_cache()
    V0, V1, loss = _one_gd_step(P, plan, B, "bf16", segment=16)
    loss_rel, g_err = _bf16_error(orc, V0, V1, loss, _samples(B, 3))
    print(f"1M gates, bf16 activations, recompute 16: loss max rel {loss_rel:.3g}, "
          f"dL/dV err / sum|terms| {g_err:.3g}")
    assert loss_rel <= BOUNDS["bf16"][0] and g_err <= BOUNDS["bf16"][1]


def test_1m_verification_and_dedup(gpu, c1m):
    P, inst, plan, orc, B = c1m
    _check_verification(P, inst, plan, orc, B, 2e-5, 8)
