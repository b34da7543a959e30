"""Oracle of the learned warm start's network (not in the paper).

Test infrastructure only (see ``oracle/__init__``).

The network, its loss and its optimiser, written out in FP64 numpy from
their textbook definitions:

  xn = (x - in_mean) / in_std
  a1 = xn W1^T + b1,  h1 = GELU(a1)
  a2 = h1 W2^T + b2,  h2 = GELU(a2)
  y  = h2 W3^T + b3                                   (normalised prediction)
  L  = (1 / (B d_out)) sum (y - (t - out_mean) / out_std)^2
  GELU(a) = a Phi(a) = a (1 + erf(a / sqrt 2)) / 2,
  GELU'(a) = Phi(a) + a phi(a)
  Adam (Kingma & Ba 2015): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
      w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)

The backward pass is the chain rule applied layer by layer (no automatic
differentiation).  Pins (tests/test_oracle_mlp.py): central finite
differences of L for every parameter block; GELU at points with known
values (Phi(1) = 0.8413447460685429) and its limits; Adam's first step
equals -lr sign(g) up to eps; the BF16 rounding helper on exact ties.

``bf16=True`` reproduces where the tensor-core path rounds its operands to
BF16 (round to nearest even): the normalised input, the three weight
matrices, the hidden activations fed to the next product, and the loss and
pre-activation gradients fed to the backward products; everything else stays
FP64.  It lets a GPU comparison isolate accumulation-order differences.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def bf16_round(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64).reshape(f.shape)


def gelu(a):
    return 0.5 * a * (1.0 + erf(a / SQRT2))


def gelu_d(a):
    return 0.5 * (1.0 + erf(a / SQRT2)) + a * INV_SQRT_2PI * np.exp(-0.5 * a * a)


def unflatten(p, d_in, d_h, d_out):
    """Logical parameter vector -> (W1, b1, W2, b2, W3, b3)."""
    p = np.asarray(p, dtype=np.float64)
    sizes = [d_h * d_in, d_h, d_h * d_h, d_h, d_out * d_h, d_out]
    parts = np.split(p, np.cumsum(sizes)[:-1])
    return (parts[0].reshape(d_h, d_in), parts[1], parts[2].reshape(d_h, d_h), parts[3],
            parts[4].reshape(d_out, d_h), parts[5])


def flatten(W1, b1, W2, b2, W3, b3):
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])


def _r(a, on):
    return bf16_round(a) if on else a


def forward(p, X, dims, norm, bf16=False):
    """Normalised prediction y and the cache of the backward pass."""
    d_in, d_h, d_out = dims
    in_mean, in_std = norm[0], norm[1]
    W1, b1, W2, b2, W3, b3 = unflatten(p, d_in, d_h, d_out)
    xn = _r((np.asarray(X, dtype=np.float64) - in_mean) / in_std, bf16)
    W1r, W2r, W3r = _r(W1, bf16), _r(W2, bf16), _r(W3, bf16)
    a1 = xn @ W1r.T + b1
    h1 = _r(gelu(a1), bf16)
    a2 = h1 @ W2r.T + b2
    h2 = _r(gelu(a2), bf16)
    y = h2 @ W3r.T + b3
    return y, (xn, a1, h1, a2, h2, W2r, W3r)


def predict(p, X, dims, norm):
    """De-normalised prediction out_mean + out_std * y."""
    y, _ = forward(p, X, dims, norm)
    return norm[2] + norm[3] * y


def loss_and_grad(p, X, T, dims, norm, bf16=False):
    """Mean squared error of the normalised outputs and its gradient (logical layout)."""
    d_in, d_h, d_out = dims
    y, (xn, a1, h1, a2, h2, W2r, W3r) = forward(p, X, dims, norm, bf16)
    B = y.shape[0]
    tn = (np.asarray(T, dtype=np.float64) - norm[2]) / norm[3]
    d = y - tn
    L = float((d * d).sum() / (B * d_out))
    dy = 2.0 * d / (B * d_out)
    dyr = _r(dy, bf16)
    gW3 = dyr.T @ h2
    gb3 = dy.sum(axis=0)
    da2 = (dyr @ W3r) * gelu_d(a2)
    da2r = _r(da2, bf16)
    gW2 = da2r.T @ h1
    gb2 = da2.sum(axis=0)
    da1 = (da2r @ W2r) * gelu_d(a1)
    gW1 = _r(da1, bf16).T @ xn
    gb1 = da1.sum(axis=0)
    return L, flatten(gW1, gb1, gW2, gb2, gW3, gb3)


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update at step t (1-based); returns (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
