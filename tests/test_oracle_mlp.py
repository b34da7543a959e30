"""Pins of the warm-start network oracle (oracle/mlp.py), CPU only."""
import math

import numpy as np
import pytest

from oracle import mlp


def small(seed=0, d_in=7, d_h=5, d_out=4, B=6):
    rng = np.random.default_rng(seed)
    n = d_h * d_in + d_h + d_h * d_h + d_h + d_out * d_h + d_out
    p = rng.normal(0, 0.5, n)
    X = rng.normal(0, 1, (B, d_in))
    T = rng.normal(0, 1, (B, d_out))
    norm = (rng.normal(0, 0.1, d_in), rng.uniform(0.5, 2, d_in), rng.normal(0, 0.1, d_out),
            rng.uniform(0.5, 2, d_out))
    return p, X, T, (d_in, d_h, d_out), norm


def test_gelu_known_values():
    # GELU(1) = Phi(1); GELU(0) = 0; GELU'(0) = 1/2; GELU(-x) = GELU(x) - x
    assert mlp.gelu(np.array(1.0)) == pytest.approx(0.8413447460685429, abs=1e-15)
    assert mlp.gelu(np.array(0.0)) == 0.0
    assert mlp.gelu_d(np.array(0.0)) == pytest.approx(0.5, abs=1e-16)
    x = np.linspace(-3, 3, 13)
    np.testing.assert_allclose(mlp.gelu(-x), mlp.gelu(x) - x, atol=1e-15)
    # limits: identity for large positive, zero for large negative arguments
    assert mlp.gelu(np.array(12.0)) == pytest.approx(12.0, abs=1e-12)
    assert abs(mlp.gelu(np.array(-12.0))) < 1e-12


def test_gelu_derivative_by_differences():
    x = np.linspace(-4, 4, 41)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_d(x), fd, atol=1e-9)


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_central_differences(seed):
    p, X, T, dims, norm = small(seed)
    L, g = mlp.loss_and_grad(p, X, T, dims, norm)
    fd = np.zeros_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        h = 1e-6 * max(1.0, abs(p[i]))
        e[i] = h
        fd[i] = (mlp.loss_and_grad(p + e, X, T, dims, norm)[0] - mlp.loss_and_grad(p - e, X, T, dims, norm)[0]) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)


def test_loss_zero_at_targets_and_prediction_denormalised():
    p, X, T, dims, norm = small(2)
    y, _ = mlp.forward(p, X, dims, norm)
    T0 = norm[2] + norm[3] * y
    L, g = mlp.loss_and_grad(p, X, T0, dims, norm)
    assert L < 1e-28
    assert np.abs(g).max() < 1e-14
    np.testing.assert_allclose(mlp.predict(p, X, dims, norm), T0, rtol=1e-15)


def test_flatten_roundtrip_and_shapes():
    p, X, T, dims, norm = small(3)
    parts = mlp.unflatten(p, *dims)
    assert parts[0].shape == (dims[1], dims[0]) and parts[4].shape == (dims[2], dims[1])
    np.testing.assert_array_equal(mlp.flatten(*parts), p)


def test_adam_first_step_is_signed_learning_rate():
    g = np.array([3.0, -0.2, 1e-3, -40.0])
    p0 = np.ones(4)
    p1, m, v = mlp.adam_step(p0, g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    # m_hat = g, v_hat = g^2 at t = 1, so the step is -lr g / (|g| + eps)
    np.testing.assert_allclose(p1 - p0, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(np.abs(p1 - p0), 0.01, rtol=1e-4)


def test_bf16_rounding_ties_and_exact_values():
    u = 2.0 ** -7  # BF16 spacing at 1
    vals = np.array([1.0, 1.0 + u / 2, 1.0 + 1.5 * u, 1.0 + u / 4, -3.0, 0.0, 1.0 + 0.75 * u])
    want = np.array([1.0, 1.0, 1.0 + 2 * u, 1.0, -3.0, 0.0, 1.0 + u])
    np.testing.assert_array_equal(mlp.bf16_round(vals), want)
    x = np.random.default_rng(0).normal(size=1000)
    r = mlp.bf16_round(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -8 * (1 + 1e-7))


def test_bf16_emulation_stays_close():
    p, X, T, dims, norm = small(4, d_in=16, d_h=8, d_out=6, B=10)
    L, g = mlp.loss_and_grad(p, X, T, dims, norm)
    Lb, gb = mlp.loss_and_grad(p, X, T, dims, norm, bf16=True)
    assert abs(Lb - L) <= 0.05 * L
    assert np.linalg.norm(gb - g) <= 0.05 * np.linalg.norm(g)
