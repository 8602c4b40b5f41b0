"""FP64 oracle of the learned proposal network (test infrastructure only).

The paper has no learned component; this restates, in plain numpy, what the
library's proposal network computes so its CUDA kernels can be checked:

* MLP z (n_in) -> GELU(z W1^T + b1) -> GELU(. W2^T + b2) -> . W3^T + b3 = y
  (n_out logits, one per primary input), GELU in its exact form
  x Phi(x) = x (1 + erf(x / sqrt 2)) / 2 (erf from scipy).
* Loss: binary cross-entropy with logits against the solution bits t, averaged
  over samples and outputs: mean(softplus(y) - t y).
* Gradients by the chain rule (written out below, layer by layer).
* IMLE selection (Li and Malik, 2018): for every target, among its K candidate
  noise vectors pick the one whose output has the least summed BCE to it
  (first index on ties).
* The magnitude of the backward pass (every factor in absolute value), which
  scales the rounding error of a low-precision evaluation of the gradient.
* The noise z ~ N(0, I): Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
  blocks turned into normals by the Box-Muller transform.

Parameter vector order: W1 [h][n_in], b1 [h], W2 [h][h], b2 [h], W3 [n_out][h], b3 [n_out].
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

SQRT2 = np.sqrt(2.0)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / SQRT2))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / SQRT2)) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def unpack(theta, n_in, h, n_out):
    shapes = [(h, n_in), (h,), (h, h), (h,), (n_out, h), (n_out,)]
    out, o = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append(np.asarray(theta[o:o + n], dtype=np.float64).reshape(s))
        o += n
    assert o == len(theta)
    return out


def n_params(n_in, h, n_out):
    return h * n_in + h + h * h + h + n_out * h + n_out


def forward(theta, Z, n_in, h, n_out):
    W1, b1, W2, b2, W3, b3 = unpack(theta, n_in, h, n_out)
    Z = np.asarray(Z, dtype=np.float64)
    p1 = Z @ W1.T + b1
    h1 = gelu(p1)
    p2 = h1 @ W2.T + b2
    h2 = gelu(p2)
    y = h2 @ W3.T + b3
    return y, (Z, p1, h1, p2, h2)


def bce_terms(y, t):
    """softplus(y) - t y, elementwise, computed stably."""
    return np.maximum(y, 0.0) - t * y + np.log1p(np.exp(-np.abs(y)))


def loss(theta, Z, T, n_in, h, n_out):
    y, _ = forward(theta, Z, n_in, h, n_out)
    return bce_terms(y, T).mean()


def grad(theta, Z, T, n_in, h, n_out):
    """Gradient of the mean BCE loss w.r.t. the parameter vector."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, n_in, h, n_out)
    y, (Z, p1, h1, p2, h2) = forward(theta, Z, n_in, h, n_out)
    dy = (1.0 / (1.0 + np.exp(-y)) - T) / y.size
    dW3, db3 = dy.T @ h2, dy.sum(0)
    da2 = (dy @ W3) * gelu_grad(p2)
    dW2, db2 = da2.T @ h1, da2.sum(0)
    da1 = (da2 @ W2) * gelu_grad(p1)
    dW1, db1 = da1.T @ Z, da1.sum(0)
    return np.concatenate([a.ravel() for a in (dW1, db1, dW2, db2, dW3, db3)])


def grad_magnitude(theta, Z, D, n_in, h, n_out):
    """The backward pass of `grad` with every factor in absolute value, seeded with
    |D| [S][n_out] in place of dL/dy: the sums of absolute terms behind each gradient
    entry.  With D = dL/dy it bounds |grad| entry by entry (triangle inequality), with
    equality when every term is non-negative."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, n_in, h, n_out)
    _, (Z, p1, h1, p2, h2) = forward(theta, Z, n_in, h, n_out)
    dy = np.abs(np.asarray(D, dtype=np.float64))
    dW3, db3 = dy.T @ np.abs(h2), dy.sum(0)
    da2 = (dy @ np.abs(W3)) * np.abs(gelu_grad(p2))
    dW2, db2 = da2.T @ np.abs(h1), da2.sum(0)
    da1 = (da2 @ np.abs(W2)) * np.abs(gelu_grad(p1))
    dW1, db1 = da1.T @ np.abs(Z), da1.sum(0)
    return np.concatenate([a.ravel() for a in (dW1, db1, dW2, db2, dW3, db3)])


def output_grad(theta, Z, T, n_in, h, n_out):
    """dL/dy of the mean BCE: (sigmoid(y) - t) / (S n_out)."""
    y, _ = forward(theta, Z, n_in, h, n_out)
    return (1.0 / (1.0 + np.exp(-y)) - T) / y.size


def noise(rows, n_in, seed, rnd):
    """z [rows][n_in]: the Philox4x32-10 block at counter (row, c, rnd, 1) under key
    (seed low word, seed high word) gives z[row][4c .. 4c+3]; each pair of words (x, y)
    becomes u1 = ((x >> 8) + 1) / 2^24, u2 = (y >> 8) / 2^24 and the Box-Muller pair
    r cos(2 pi u2), r sin(2 pi u2) with r = sqrt(-2 ln u1)."""
    from .sampler import philox4x32_10
    key = [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF]
    z = np.zeros((rows, n_in))
    for r in range(rows):
        for c in range((n_in + 3) // 4):
            o = philox4x32_10([r, c, rnd, 1], key)
            vals = []
            for x, y in ((o[0], o[1]), (o[2], o[3])):
                u1 = ((x >> 8) + 1) / 16777216.0
                u2 = (y >> 8) / 16777216.0
                rad = np.sqrt(-2.0 * np.log(u1))
                vals += [rad * np.cos(2.0 * np.pi * u2), rad * np.sin(2.0 * np.pi * u2)]
            for i, v in enumerate(vals):
                if 4 * c + i < n_in:
                    z[r, 4 * c + i] = v
    return z


def imle_select(theta, Zc, T, K, n_in, h, n_out):
    """Zc: [S*K][n_in] candidates (candidate k of target s at row s*K + k); T: [S][n_out].
    Returns (choice [S], distances [S*K])."""
    y, _ = forward(theta, Zc, n_in, h, n_out)
    S = T.shape[0]
    d = bce_terms(y, np.repeat(T, K, axis=0)).sum(1)
    return d.reshape(S, K).argmin(1), d


def init_params(n_in, h, n_out, seed):
    """PyTorch nn.Linear default: U(-1/sqrt(fan_in), 1/sqrt(fan_in)) for weights and biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((h, n_in), (h, h), (n_out, h)):
        k = 1.0 / np.sqrt(fan_in)
        parts.append(rng.uniform(-k, k, fan_out * fan_in))
        parts.append(rng.uniform(-k, k, fan_out))
    return np.concatenate(parts)
