"""Pins for the FP64 tolerance-network oracle (oracle/mlp.py)."""
import math

import numpy as np

import synth
from oracle import mlp


def _data(n=64, seed=0):
    rng = np.random.default_rng(seed)
    s = np.exp(rng.uniform(0, math.log(16), n))
    U = mlp.features(s, rng.uniform(0, 2 * math.pi, n), (1 / s) * np.exp(rng.normal(0, 0.3, n)),
                     rng.random(n), rng.random(n))
    r = np.abs(rng.normal(0, 0.6 * s))
    return U, r


def test_param_layout():
    th = synth.mlp_init(0)
    assert th.size == synth.mlp_param_count() == 8769
    assert sum(W.size + b.size for W, b in mlp.unpack(th)) == th.size


def test_gradient_matches_central_differences():
    U, r = _data()
    th = synth.mlp_init(1).astype(np.float64) + np.random.default_rng(2).normal(0, 0.05, 8769)
    g = mlp.grad(th, U, r, 0.9)
    rng = np.random.default_rng(3)
    idx = np.concatenate([rng.choice(8769, 120, replace=False), [8768, 8767, 0, 319, 384]])
    h = 1e-6
    for k in idx:
        e = np.zeros_like(th)
        e[k] = h
        fd = (mlp.loss(th + e, U, r, 0.9) - mlp.loss(th - e, U, r, 0.9)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, k


def test_gelu_and_softplus_identities():
    x = np.linspace(-8, 8, 101)
    # Phi(x) + Phi(-x) = 1  =>  GELU(x) - GELU(-x) = x
    assert np.allclose(mlp.gelu(x) - mlp.gelu(-x), x, atol=1e-14)
    assert mlp.gelu(0.0) == 0.0
    assert np.allclose(mlp.softplus(x) - mlp.softplus(-x), x, atol=1e-13)
    assert abs(mlp.softplus(0.0) - math.log(2.0)) < 1e-15


def test_pinball_minimiser_is_the_quantile():
    """With a constant prediction the pinball loss is minimised at the
    q-quantile of the residuals: the bias gradient changes sign there."""
    rng = np.random.default_rng(5)
    r = rng.exponential(2.0, 2001)
    q = 0.9
    th = np.zeros(8769)
    U = np.zeros((r.size, 5))
    # eps = softplus(b4) + 0.25; move b4 across the empirical quantile
    target = np.quantile(r, q, method="inverted_cdf")
    b_at = math.log(math.expm1(target - 0.25))
    th[-1] = b_at - 1e-3
    g_lo = mlp.grad(th, U, r, q)[-1]
    th[-1] = b_at + 1e-3
    g_hi = mlp.grad(th, U, r, q)[-1]
    assert g_lo < 0 < g_hi


def test_adam_first_step_is_signed_learning_rate():
    g = np.array([3.0, -0.5, 1e-3, -7.0])
    th, m, v = mlp.adam_step(np.zeros(4), np.zeros(4), np.zeros(4), g, 1, 1e-3)
    assert np.allclose(th, -1e-3 * np.sign(g), rtol=1e-4)
