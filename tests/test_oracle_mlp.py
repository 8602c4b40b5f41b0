"""Pins of the proposal-network oracle: closed forms, central differences, brute-force IMLE."""
import math

import numpy as np
import pytest

from oracle import mlp as M


def test_gelu_closed_forms():
    assert M.gelu(np.array(0.0)) == 0.0
    assert abs(M.gelu_grad(np.array(0.0)) - 0.5) < 1e-15
    x = np.array([-3.0, -0.5, 0.7, 4.0])
    phi = np.array([0.5 * (1 + math.erf(v / math.sqrt(2))) for v in x])
    np.testing.assert_allclose(M.gelu(x), x * phi, rtol=1e-14)
    h = 1e-6
    np.testing.assert_allclose(M.gelu_grad(x), (M.gelu(x + h) - M.gelu(x - h)) / (2 * h), rtol=1e-8)


def test_bce_closed_form():
    y = np.array([-5.0, -1.0, 0.0, 2.0, 5.0])
    for t in (0.0, 1.0):
        p = 1 / (1 + np.exp(-y))
        direct = -(t * np.log(p) + (1 - t) * np.log(1 - p))
        np.testing.assert_allclose(M.bce_terms(y, t), direct, rtol=1e-10)
    assert abs(M.bce_terms(np.array(0.0), 1.0) - math.log(2)) < 1e-15
    # far tails: softplus(y) - t y -> |y| for the wrong label, -> 0 for the right one
    assert abs(M.bce_terms(np.array(40.0), 0.0) - 40.0) < 1e-12
    assert M.bce_terms(np.array(40.0), 1.0) < 1e-17


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_central_differences(seed):
    n_in, h, n_out, S = 5, 7, 6, 4
    rng = np.random.default_rng(seed)
    theta = M.init_params(n_in, h, n_out, seed) * 2.0
    Z = rng.normal(size=(S, n_in))
    T = rng.integers(0, 2, (S, n_out)).astype(np.float64)
    g = M.grad(theta, Z, T, n_in, h, n_out)
    eps = 1e-6
    fd = np.zeros_like(theta)
    for i in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd[i] = (M.loss(tp, Z, T, n_in, h, n_out) - M.loss(tm, Z, T, n_in, h, n_out)) / (2 * eps)
    assert np.abs(fd - g).max() <= 1e-6 * np.abs(g).max()


def test_imle_select_is_brute_force_argmin():
    n_in, h, n_out, S, K = 4, 6, 5, 3, 8
    rng = np.random.default_rng(3)
    theta = M.init_params(n_in, h, n_out, 3)
    Zc = rng.normal(size=(S * K, n_in))
    T = rng.integers(0, 2, (S, n_out)).astype(np.float64)
    choice, d = M.imle_select(theta, Zc, T, K, n_in, h, n_out)
    for s in range(S):
        losses = [M.loss(theta, Zc[s * K + k][None], T[s][None], n_in, h, n_out) * n_out for k in range(K)]
        assert choice[s] == int(np.argmin(losses))
        np.testing.assert_allclose(d[s * K:(s + 1) * K], losses, rtol=1e-12)


def test_param_layout():
    assert M.n_params(64, 256, 2000) == 64 * 256 + 256 + 256 * 256 + 256 + 2000 * 256 + 2000
    th = np.arange(M.n_params(2, 3, 4), dtype=float)
    W1, b1, W2, b2, W3, b3 = M.unpack(th, 2, 3, 4)
    assert W1.shape == (3, 2) and W1[0, 1] == 1 and b1[0] == 6 and W3.shape == (4, 3) and b3[-1] == th[-1]


def test_grad_magnitude_bounds_and_equals_when_terms_are_positive():
    """With dL/dy as seed the magnitude bounds |grad| entry by entry; with every weight, bias
    and input positive (so every pre-activation and GELU' > 0) and every target 0 (so dL/dy > 0)
    all terms are positive and the magnitude equals the gradient."""
    n_in, h, n_out, S = 5, 7, 6, 4
    rng = np.random.default_rng(5)
    theta = M.init_params(n_in, h, n_out, 5) * 2.0
    Z = rng.normal(size=(S, n_in))
    T = rng.integers(0, 2, (S, n_out)).astype(np.float64)
    g = M.grad(theta, Z, T, n_in, h, n_out)
    gm = M.grad_magnitude(theta, Z, M.output_grad(theta, Z, T, n_in, h, n_out), n_in, h, n_out)
    assert (gm >= np.abs(g) * (1 - 1e-12)).all() and (gm > np.abs(g) * (1 + 1e-9)).any()
    thp, Zp, T0 = np.abs(theta), np.abs(Z), np.zeros((S, n_out))
    g = M.grad(thp, Zp, T0, n_in, h, n_out)
    gm = M.grad_magnitude(thp, Zp, M.output_grad(thp, Zp, T0, n_in, h, n_out), n_in, h, n_out)
    assert (g > 0).all()
    np.testing.assert_allclose(gm, g, rtol=1e-12)


def test_noise_is_standard_normal_and_uses_the_stated_blocks():
    """Moments of the Box-Muller noise, and its first entries re-derived from the pinned
    Philox block function (counter (row, group, round, 1))."""
    import oracle
    z = M.noise(400, 64, 7, 3)
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1) < 0.02
    assert abs(((z - z.mean()) ** 3).mean()) < 0.05 and abs((z ** 4).mean() - 3) < 0.15
    o = oracle.philox4x32_10([2, 1, 3, 1], [7, 0])
    r = math.sqrt(-2 * math.log(((o[2] >> 8) + 1) / 2 ** 24))
    assert abs(z[2, 6] - r * math.cos(2 * math.pi * (o[3] >> 8) / 2 ** 24)) < 1e-12
    assert np.array_equal(M.noise(5, 10, 7, 3), z[:5, :10])
