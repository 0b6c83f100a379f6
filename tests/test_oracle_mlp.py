"""Pins of the oracle's MLP (CPU only): gradients against central differences, a linear layer
against the closed-form least-squares gradient, Adam's first step against its closed form."""
import numpy as np

from oracle import mlp
from paper_2410_18740_gb300 import inputs


def _setup(seed, n_in, width, depth, n_out, B):
    rng = inputs.rng_for(seed)
    n = mlp.param_count(n_in, width, depth, n_out)
    p = rng.uniform(-0.5, 0.5, size=n)
    x = rng.standard_normal((B, n_in))
    t = rng.standard_normal((B, n_out))
    return p, x, t


def test_gradient_matches_central_differences():
    dims = (3, 7, 3, 2)
    p, x, t = _setup(0, *dims, B=5)
    _, g = mlp.loss_and_grad(p, x, t, *dims)
    h = 1e-6
    rng = inputs.rng_for(1)
    for j in rng.choice(p.size, size=40, replace=False):
        e = np.zeros_like(p)
        e[j] = h
        lp, _ = mlp.loss_and_grad(p + e, x, t, *dims)
        lm, _ = mlp.loss_and_grad(p - e, x, t, *dims)
        assert abs((lp - lm) / (2 * h) - g[j]) <= 1e-7 * max(1.0, abs(g[j]))


def test_linear_layer_gradient_closed_form():
    """depth 0: y = x W^T + b, loss = |y - t|^2 / (B n_out): dW = 2 (y - t)^T x / (B n_out)."""
    n_in, n_out, B = 4, 3, 6
    p, x, t = _setup(2, n_in, 1, 0, n_out, B)
    W = p[: n_in * n_out].reshape(n_out, n_in)
    b = p[n_in * n_out:]
    r = x @ W.T + b - t
    loss, g = mlp.loss_and_grad(p, x, t, n_in, 1, 0, n_out)
    assert abs(loss - np.sum(r * r) / (B * n_out)) < 1e-14
    assert np.abs(g[: n_in * n_out] - (2 * r.T @ x / (B * n_out)).reshape(-1)).max() < 1e-14
    assert np.abs(g[n_in * n_out:] - 2 * r.sum(axis=0) / (B * n_out)).max() < 1e-14


def test_adam_first_step_closed_form():
    rng = inputs.rng_for(3)
    p = rng.standard_normal(50)
    g = rng.standard_normal(50)
    z = np.zeros(50)
    p1, m, v = mlp.adam_step(p, z, z, g, 1, lr=1e-3)
    assert np.abs(p1 - (p - 1e-3 * g / (np.abs(g) + 1e-8))).max() < 1e-15
    assert np.abs(m - 0.1 * g).max() < 1e-15 and np.abs(v - 0.001 * g * g).max() < 1e-15


def test_training_fits_a_smooth_target():
    """A few hundred Adam steps reduce the loss on y = sin(x1) + x2^2 by two orders."""
    rng = inputs.rng_for(4)
    dims = (2, 32, 2, 1)
    n = mlp.param_count(*dims)
    p = np.concatenate([np.concatenate([rng.uniform(-1, 1, a * b) * np.sqrt(6.0 / a), np.zeros(b)])
                        for a, b in mlp.layer_sizes(*dims)])
    assert p.size == n
    x = rng.uniform(-1, 1, (256, 2))
    t = (np.sin(2 * x[:, 0]) + x[:, 1] ** 2)[:, None]
    m = np.zeros(n)
    v = np.zeros(n)
    l0, _ = mlp.loss_and_grad(p, x, t, *dims)
    for s in range(1, 401):
        _, g = mlp.loss_and_grad(p, x, t, *dims)
        p, m, v = mlp.adam_step(p, m, v, g, s, lr=1e-2)
    l1, _ = mlp.loss_and_grad(p, x, t, *dims)
    assert l1 < 1e-2 * l0
