"""Proposal network on the GPU (tcgen05 GEMMs) against the FP64 oracle.

Inputs are seeded (weights from workloads.mlp_params, noise rows from
workloads.normal_logits), set on the GPU and given to the oracle; the GPU rounds
weights, activations and the backward's adjoints to BF16 and accumulates in FP32,
the oracle runs in FP64 on the same BF16-rounded weights and noise.  Bounds:
* logits within 4 * 2^-8 of the magnitude sum |H2| |W3|^T + |b3| (two BF16
  roundings feed the last layer);
* every gradient entry within 8 * 2^-8 of the sum of absolute terms behind it
  (oracle.mlp.grad_magnitude seeded with |dL/dy|: the BF16 roundings of dL/dy,
  of both hidden adjoints and of the activations they meet), plus the effect of
  the logits' own bound on dL/dy = (sigmoid(y) - t) / N, i.e. the magnitude pass
  seeded with sigmoid'(y) times that bound;
* the optimiser (FP32) within a few FP32 roundings of FP64 Adam on the same
  gradients.
"""
import numpy as np
import pytest

from oracle import mlp as M
from workloads import mlp_params, normal_logits, normal_vector

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _bf16(x):
    return torch.tensor(np.asarray(x, dtype=np.float32)).to(torch.bfloat16).double().numpy()


def _rounded_theta(theta, n_in, h, n_out):
    """Weights as the GPU uses them (bf16), biases as they are (fp32)."""
    W1, b1, W2, b2, W3, b3 = M.unpack(theta, n_in, h, n_out)
    return np.concatenate([_bf16(W1).ravel(), b1, _bf16(W2).ravel(), b2, _bf16(W3).ravel(), b3])


def _keys(bits):
    S, n = bits.shape
    kw = (n + 31) // 32
    words = np.zeros((S, kw), np.uint32)
    for i in range(n):
        words[:, i // 32] |= bits[:, i].astype(np.uint32) << np.uint32(i % 32)
    return torch.tensor(words.view(np.int32))


def _mlp(n_in, h, n_out, max_rows, seed):
    """A network holding the seeded parameters mlp_params(..., seed); returns it and them."""
    import paper_2502_08673_b300 as P
    mlp = P.Mlp.create(n_in, h, n_out, max_rows=max_rows, seed=0)
    theta = mlp_params(n_in, h, n_out, seed)
    mlp.set_params(theta)
    return mlp, theta.astype(np.float64)


def _noise(rows, n_in, seed, device):
    """Seeded noise rows as the GPU takes them (bf16) and their exact values."""
    z = torch.tensor(normal_logits(rows, n_in, seed)).to(torch.bfloat16).to(device)
    return z, z.double().cpu().numpy()


@pytest.mark.parametrize("n_out", [64, 200, 2000])
def test_forward_matches_oracle(gpu, n_out):
    n_in, h, R = 64, 256, 300
    mlp, theta = _mlp(n_in, h, n_out, 512, seed=3)
    z, zr = _noise(R, n_in, 11, gpu)
    V = mlp.forward(z, tau=1.5)
    torch.cuda.synchronize()
    assert mlp.status() == 0
    th = _rounded_theta(theta, n_in, h, n_out)
    y, (_, p1, h1, p2, h2) = M.forward(th, zr, n_in, h, n_out)
    W3 = M.unpack(th, n_in, h, n_out)[4]
    mag = np.abs(h2) @ np.abs(W3).T + np.abs(theta[-n_out:])
    got = V.cpu().double().numpy().T / 1.5
    assert (np.abs(got - y) <= 4 * 2 ** -8 * mag + 1e-6).all(), float(np.abs(got - y).max())


def test_forward_at_the_1m_gate_workload_size(gpu):
    """The proposal of the 1M-gate workload (50,000 inputs) at its batch of 8,192 rows, as the
    sampler runs it (noise drawn on the device, tau = 2, FP32 logits written into V [n][B]):
    sampled rows (both ends of every 128-row tile boundary case, and random ones) against the
    FP64 oracle on the same BF16 noise and weights, within the forward bound above."""
    n_in, h, n_out, R, tau = 64, 256, 50000, 8192, 2.0
    mlp, theta = _mlp(n_in, h, n_out, R, seed=13)
    z = mlp.draw_noise(R, seed=4, round_=1)
    V = torch.empty((n_out, R), dtype=torch.float32, device=gpu)
    mlp.forward(z, tau=tau, V=V)
    torch.cuda.synchronize()
    assert mlp.status() == 0
    idx = np.array(sorted(set([0, 1, 127, 128, 4095, 4096, R - 1] + list(np.random.default_rng(0).integers(0, R, 17)))))
    zr = z[torch.tensor(idx, device=gpu)].double().cpu().numpy()
    th = _rounded_theta(theta, n_in, h, n_out)
    y, (_, _, _, _, h2) = M.forward(th, zr, n_in, h, n_out)
    W3 = M.unpack(th, n_in, h, n_out)[4]
    mag = np.abs(h2) @ np.abs(W3).T + np.abs(theta[-n_out:])
    got = V[:, torch.tensor(idx, device=gpu)].cpu().double().numpy().T / tau
    err = np.abs(got - y)
    print(f"proposal at 50,000 outputs: max |y - y*| / bound = {float((err / (4 * 2 ** -8 * mag + 1e-6)).max()):.3g}")
    assert (err <= 4 * 2 ** -8 * mag + 1e-6).all(), float(err.max())
    assert torch.isfinite(V).all()


def test_noise_matches_oracle(gpu):
    """sat_mlp_draw_noise = the oracle's Philox4x32-10 + Box-Muller noise, rounded to BF16
    (the GPU's FP32 log/sincos may land on the other side of a BF16 rounding boundary:
    at most one BF16 step, rarely); reproducible; standard normal moments."""
    import paper_2502_08673_b300 as P
    n_in, R = 64, 300
    mlp = P.Mlp.create(n_in, 256, 64, max_rows=20000, seed=0)
    z = mlp.draw_noise(R, seed=11, round_=5)
    torch.cuda.synchronize()
    ref = M.noise(R, n_in, 11, 5)
    got = z.double().cpu().numpy()
    assert (np.abs(got - ref) <= 2 ** -7 * np.abs(ref) + 2 ** -30).all()
    assert (got == _bf16(ref)).mean() > 0.99
    assert torch.equal(mlp.draw_noise(R, seed=11, round_=5), z)
    zz = mlp.draw_noise(20000, seed=11).float()
    assert abs(zz.mean().item()) < 0.01 and abs(zz.std().item() - 1) < 0.01


def test_loss_and_gradient_match_oracle(gpu):
    n_in, h, n_out, S = 64, 256, 200, 384
    mlp, theta = _mlp(n_in, h, n_out, 1024, seed=5)
    rng = np.random.default_rng(0)
    bits = rng.integers(0, 2, (S, n_out))
    keys = _keys(bits).to(gpu)
    z, zr = _noise(S, n_in, 2, gpu)
    loss, g = mlp.loss_grad(z, keys)
    th = _rounded_theta(theta, n_in, h, n_out)
    T = bits.astype(np.float64)
    assert abs(loss - M.loss(th, zr, T, n_in, h, n_out)) < 2e-3 * abs(loss) + 1e-6
    gref = M.grad(th, zr, T, n_in, h, n_out)
    # per-entry bound: BF16 roundings in the backward, and the logits' bound carried into dL/dy
    y, (_, _, _, _, h2) = M.forward(th, zr, n_in, h, n_out)
    W3 = M.unpack(th, n_in, h, n_out)[4]
    ey = 4 * 2 ** -8 * (np.abs(h2) @ np.abs(W3).T + np.abs(theta[-n_out:]))
    sig = 1.0 / (1.0 + np.exp(-y))
    dy = M.output_grad(th, zr, T, n_in, h, n_out)
    tol = (8 * 2 ** -8 * M.grad_magnitude(th, zr, dy, n_in, h, n_out)
           + M.grad_magnitude(th, zr, sig * (1 - sig) * ey / y.size, n_in, h, n_out))
    a = g.astype(np.float64)
    ratio = np.abs(a - gref) / tol
    print(f"proposal gradient: max |g - g*| / bound = {ratio.max():.3g}")
    assert (ratio <= 1).all(), (np.argwhere(ratio > 1)[:5], ratio.max())
    sizes = [h * n_in, h, h * h, h, n_out * h, n_out]
    o = 0
    for sz in sizes:
        ga, gb = a[o:o + sz], gref[o:o + sz]
        assert ga @ gb / (np.linalg.norm(ga) * np.linalg.norm(gb)) > 0.999
        o += sz
    assert mlp.status() == 0


def test_adam_update_matches_oracle(gpu):
    """sat_mlp_apply_grad: FP32 Adam of the master weights against the oracle's FP64 Adam on
    the same seeded gradients, over 40 steps (bias corrections at t = 1..40), and the BF16
    copies used by the next forward refreshed."""
    import oracle
    n_in, h, n_out = 64, 256, 200
    mlp, theta = _mlp(n_in, h, n_out, 256, seed=9)
    lr = 1e-2
    f32 = lambda x: float(np.float32(x))  # noqa: E731  (the network's FP32 constants)
    V, m, v = theta.copy(), np.zeros_like(theta), np.zeros_like(theta)
    for t in range(1, 41):
        g = normal_vector(theta.size, seed=100 + t, scale=1e-2)
        mlp.apply_grad(torch.tensor(g, device=gpu), lr)
        oracle.adam_step(V, m, v, g.astype(np.float64), t, f32(lr), f32(0.9), f32(0.999), f32(1e-8))
        if t in (1, 2, 40):
            # each FP32 step rounds the update (a few ulps of lr) and the new weight (half an
            # ulp of |V|); the errors add up over t steps at most
            got = mlp.params().astype(np.float64)
            err = np.abs(got - V)
            tol = t * (1e-6 * lr + 2 ** -24 * np.abs(V)) + 1e-12
            print(f"proposal Adam t={t}: max |theta - theta*| / bound = {float((err / tol).max()):.3g}")
            assert (err <= tol).all(), (t, float((err / tol).max()))
    # the forward uses the updated weights (BF16 copies refreshed)
    z, zr = _noise(32, n_in, 4, gpu)
    out = mlp.forward(z)
    torch.cuda.synchronize()
    th = _rounded_theta(mlp.params().astype(np.float64), n_in, h, n_out)
    y, (_, _, _, _, h2) = M.forward(th, zr, n_in, h, n_out)
    W3 = M.unpack(th, n_in, h, n_out)[4]
    mag = np.abs(h2) @ np.abs(W3).T + np.abs(th[-n_out:])
    assert (np.abs(out.cpu().double().numpy().T - y) <= 4 * 2 ** -8 * mag + 1e-6).all()


def test_train_step_is_select_grad_apply(gpu):
    """sat_mlp_train_step = IMLE selection on its own noise draw, the loss gradient at the
    chosen rows, and sat_mlp_apply_grad with that gradient, bit for bit (two steps)."""
    n_in, h, n_out, S, K = 64, 256, 120, 48, 4
    a, _ = _mlp(n_in, h, n_out, S * K, seed=12)
    b, _ = _mlp(n_in, h, n_out, S * K, seed=12)
    bits = np.random.default_rng(3).integers(0, 2, (S, n_out))
    keys = _keys(bits).to(gpu)
    for r in range(2):
        la = a.train_step(keys, S, K, lr=1e-3, seed=6, round_=r)
        zc = b.draw_noise(S * K, seed=6, round_=r)
        _, choice = b.imle_select(zc, keys, S, K)
        rows = torch.arange(S, device=gpu) * K + choice.long()
        lb, g = b.loss_grad(zc[rows].contiguous(), keys)
        b.apply_grad(torch.tensor(g, device=gpu), 1e-3)
        torch.cuda.synchronize()
        assert la == lb
        assert np.array_equal(a.params(), b.params())


def test_imle_selection_matches_oracle(gpu):
    n_in, h, n_out, S, K = 64, 256, 120, 40, 16
    mlp, theta = _mlp(n_in, h, n_out, S * K, seed=8)
    rng = np.random.default_rng(1)
    bits = rng.integers(0, 2, (S, n_out))
    zc, zcr = _noise(S * K, n_in, 4, gpu)
    dist, choice = mlp.imle_select(zc, _keys(bits).to(gpu), S, K)
    torch.cuda.synchronize()
    th = _rounded_theta(theta, n_in, h, n_out)
    cref, dref = M.imle_select(th, zcr, bits.astype(np.float64), K, n_in, h, n_out)
    d = dist.cpu().double().numpy()
    tol = 2e-3 * np.abs(dref) + 1e-3
    assert (np.abs(d - dref) <= tol).all()
    ch = choice.cpu().numpy()
    for s in range(S):
        row = dref[s * K:(s + 1) * K]
        # the kernel's pick is the oracle's argmin, or ties with it within the distance tolerance
        assert ch[s] == cref[s] or row[ch[s]] - row[cref[s]] <= 2 * tol[s * K + cref[s]]


def test_imle_training_reduces_loss(gpu):
    import paper_2502_08673_b300 as P
    n_in, h, n_out, S, K = 64, 256, 96, 256, 8
    mlp = P.Mlp.create(n_in, h, n_out, max_rows=S * K, seed=1)
    rng = np.random.default_rng(2)
    # targets drawn from two prototypes with 5% noise: a learnable distribution
    proto = rng.integers(0, 2, (2, n_out))
    bits = proto[rng.integers(0, 2, S)] ^ (rng.random((S, n_out)) < 0.05)
    keys = _keys(bits).to(gpu)
    losses = [mlp.train_step(keys, S, K, lr=3e-3, seed=7, round_=r) for r in range(60)]
    torch.cuda.synchronize()
    assert mlp.status() == 0
    assert np.isfinite(losses).all()
    assert np.mean(losses[-5:]) < 0.5 * np.mean(losses[:5])


def test_train_on_solutions_equals_manual_steps(gpu):
    """sat_mlp_train: the targets are the solutions' primary-input bits, S of them drawn per
    step by SplitMix64 (Steele, Lea, Flood 2014) of the seed; equal, bit for bit, to
    train_step on the same batches."""
    import paper_2502_08673_b300 as P
    from workloads import tseitin_random_circuit
    text = tseitin_random_circuit(64, 640, 16, 8, seed=3).dimacs()
    cnf = P.Cnf.from_dimacs(text)
    circ = P.Circuit.build(cnf)
    plan = P.Plan.create(circ, cnf)
    sols = P.sample(circ, cnf, n_wanted=10 ** 9, batch=1024, steps=100, max_rounds=2, seed=0)
    W = sols.words()
    n = len(W)
    assert n > 10
    S, K, steps, seed = 64, 4, 5, 11
    a = P.Mlp.create(64, 256, plan.n_pi, max_rows=S * K, seed=2)
    b = P.Mlp.create(64, 256, plan.n_pi, max_rows=S * K, seed=2)
    la = a.train(plan, W, steps, S=S, K=K, lr=1e-3, seed=seed)
    pis = [int(v) - 1 for v in plan.pi_vars()]
    bits = np.array([[(int(W[s][v // 64]) >> (v % 64)) & 1 for v in pis] for s in range(n)], np.uint8)
    keys_all = _keys(bits)
    M64 = (1 << 64) - 1
    state = seed

    def nxt():
        nonlocal state
        state = (state + 0x9E3779B97F4A7C15) & M64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        return z ^ (z >> 31)

    lb = None
    for it in range(steps):
        idx = [nxt() % n for _ in range(S)]
        lb = b.train_step(keys_all[idx].contiguous().to(gpu), S, K, lr=1e-3, seed=seed, round_=it)
    torch.cuda.synchronize()
    assert a.status() == 0 and b.status() == 0
    assert np.array_equal(a.params(), b.params())
    assert la == lb
