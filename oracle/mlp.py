"""FP64 reference of the learned per-keypoint tolerance (test infrastructure only).

The paper proposes per-point tolerances as future work (Sec. 6) without a
model; this is the reading used by the library (network, features, target
and loss are the build's choices, stated here):

  features  u = (ln s, orientation / (2 pi), ln response, x / W, y / H)
  network   h1 = GELU(W1 u + b1), h2 = GELU(W2 h1 + b2), h3 = GELU(W3 h2 + b3)
            z = W4 h3 + b4,  eps = softplus(z) + 0.25 px
  GELU(x) = x Phi(x), Phi the standard normal CDF (erf form)
  target    residual r = distance of the true match from the epipolar line
            (Eq. 3), from the exact method
  loss      pinball loss at quantile q: mean over samples of
            max(q (r - eps), (q - 1) (r - eps))
  update    Adam (beta1 0.9, beta2 0.999, 1e-8)

Flat parameter layout: W1 (64,5), b1, W2 (64,64), b2, W3 (64,64), b3,
W4 (1,64), b4 - rows are output units (the layout of synth.mlp_init).
Pinned in tests/test_mlp_oracle.py by central finite differences, the GELU
and softplus reflection identities, the quantile property of the pinball
minimiser and Adam's first step.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

SIZES = ((64, 5), (64, 64), (64, 64), (1, 64))
EPS_FLOOR = 0.25


def unpack(theta):
    theta = np.asarray(theta, np.float64)
    out, k = [], 0
    for o, i in SIZES:
        W = theta[k:k + o * i].reshape(o, i)
        k += o * i
        b = theta[k:k + o]
        k += o
        out.append((W, b))
    assert k == theta.size
    return out


def features(scale, orientation, response, xn, yn):
    return np.stack([np.log(scale), orientation / (2 * np.pi), np.log(response), xn, yn], axis=1)


def gelu(x):
    return x * 0.5 * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def softplus(z):
    return np.logaddexp(0.0, z)


def forward(theta, U):
    """eps (n,), and the cache of pre-activations and activations."""
    layers = unpack(theta)
    h = np.asarray(U, np.float64)
    cache = [h]
    for li, (W, b) in enumerate(layers):
        a = h @ W.T + b
        if li < 3:
            cache.append(a)
            h = gelu(a)
            cache.append(h)
        else:
            z = a[:, 0]
    return softplus(z) + EPS_FLOOR, (cache, z)


def pinball(eps, r, q):
    d = r - eps
    return np.mean(np.maximum(q * d, (q - 1.0) * d))


def loss(theta, U, r, q):
    eps, _ = forward(theta, U)
    return pinball(eps, np.asarray(r, np.float64), q)


def grad(theta, U, r, q):
    """Analytic gradient of loss() with respect to the flat parameters."""
    layers = unpack(theta)
    eps, (cache, z) = forward(theta, U)
    r = np.asarray(r, np.float64)
    n = r.size
    # d pinball / d eps: -q where r > eps, (1 - q) where r < eps (0 at a tie)
    deps = np.where(r > eps, -q, np.where(r < eps, 1.0 - q, 0.0)) / n
    dz = deps / (1.0 + np.exp(-z))               # softplus' = sigmoid
    grads = [None] * 4
    delta = dz[:, None]                            # (n, 1)
    h_in = cache[6]                                # h3 (cache: u, a1, h1, a2, h2, a3, h3)
    grads[3] = (delta.T @ h_in, delta.sum(0))
    for li in (2, 1, 0):
        W_next = layers[li + 1][0]
        a = cache[1 + 2 * li]
        delta = (delta @ W_next) * gelu_grad(a)
        h_in = cache[2 * li]
        grads[li] = (delta.T @ h_in, delta.sum(0))
    return np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])


def adam_step(theta, m, v, g, t, lr, b1=0.9, b2=0.999, e=1e-8):
    """One Adam update (t counts from 1); returns (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + e), m, v
