"""Pins for the FP64 surrogate reference: finite differences, the library normal CDF, closed
forms of degenerate networks and of the first AdamW step.  No GPU needed."""
import math

import numpy as np
import pytest

from oracle import mlp


def _small(seed=0, dims=(7, 5, 4, 3)):
    return mlp.init_params(seed, dims)


def test_gelu_is_the_tanh_form_of_u_times_the_normal_cdf():
    special = pytest.importorskip("scipy.special")
    u = np.linspace(-6, 6, 241)
    # the tanh form stays within 1e-3 of the exact u * Phi(u) (library normal CDF)
    assert np.max(np.abs(mlp.gelu(u) - u * special.ndtr(u))) < 1e-3
    # derivative by central differences
    h = 1e-6
    fd = (mlp.gelu(u + h) - mlp.gelu(u - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(u), fd, rtol=1e-7, atol=1e-9)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.gelu(np.array([8.0]))[0] - 8.0) < 1e-12
    assert abs(mlp.gelu(np.array([-8.0]))[0]) < 1e-12
    # odd part: gelu(u) - gelu(-u) = u
    np.testing.assert_allclose(mlp.gelu(u) - mlp.gelu(-u), u, rtol=1e-14, atol=1e-14)


def test_gradients_by_central_differences():
    rng = np.random.default_rng(1)
    p = _small(1)
    x = rng.normal(size=(5, 7))
    y = rng.normal(size=(5, 3))
    _, g = mlp.loss_and_grads(p, x, y)
    h = 1e-6
    for k in mlp.NAMES:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = mlp.loss_and_grads(p, x, y)
            flat[idx] = old - h
            lm, _ = mlp.loss_and_grads(p, x, y)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (k, idx, fd, an)


def test_degenerate_networks():
    rng = np.random.default_rng(2)
    p = _small(2)
    x = rng.normal(size=(4, 7))
    for k in ("W1", "W2", "W3"):
        p[k] = np.zeros_like(p[k])
    out, _ = mlp.forward(p, x)
    np.testing.assert_array_equal(out, np.tile(p["b3"], (4, 1)))       # zero weights: bias only
    y = rng.normal(size=(4, 3))
    loss, g = mlp.loss_and_grads(p, x, y)
    np.testing.assert_allclose(g["b3"], 2 * (out - y).sum(0) / 12, rtol=1e-14)
    assert np.all(g["W1"] == 0) and np.all(g["W2"] == 0)             # no signal below W3 = 0
    assert abs(loss - np.mean((out - y) ** 2)) < 1e-15


def test_first_adamw_step_closed_form():
    rng = np.random.default_rng(3)
    p = _small(3)
    p0 = {k: v.copy() for k, v in p.items()}
    g = {k: rng.normal(size=v.shape) for k, v in p.items()}
    opt = mlp.AdamW(lr=1e-2, weight_decay=0.1, eps=1e-12)
    opt.step(p, g)
    for k in mlp.NAMES:
        # after one step mhat = g and vhat = g^2, so the update is lr * (sign(g) + wd * w)
        np.testing.assert_allclose(p[k], p0[k] - 1e-2 * (np.sign(g[k]) + 0.1 * p0[k]), rtol=1e-9, atol=1e-12)


def test_training_lowers_the_loss_on_a_learnable_target():
    rng = np.random.default_rng(4)
    dims = (8, 16, 16, 2)
    p = mlp.init_params(4, dims)
    x = rng.normal(size=(64, 8))
    y = np.stack([np.tanh(x[:, 0]), x[:, 1] * x[:, 2]], axis=1)
    opt = mlp.AdamW(lr=1e-2)
    l0, _ = mlp.loss_and_grads(p, x, y)
    for _ in range(200):
        _, g = mlp.loss_and_grads(p, x, y)
        opt.step(p, g)
    l1, _ = mlp.loss_and_grads(p, x, y)
    assert l1 < 0.2 * l0


def test_ood_score():
    mean = np.array([1.0, -1.0])
    std = np.array([2.0, 0.0])
    s = mlp.ood_score(np.array([[1.0, -1.0], [5.0, 1.0]]), mean, std)
    np.testing.assert_allclose(s, [0.0, (4.0 + 4.0) / 2])
