"""FP64 oracle of the surrogate network (test infrastructure).

The surrogate maps a source-receiver geometry (z_s, z_r, D) to, for up to two solutions
(sorted by travel time), an existence logit and five regression targets (launch angle,
receive angle, travel time, path length, amplitude; the normalisation is stated with
rp_surrogate_encode in include/rp.h).  Network: 3 -> 256 -> 256 -> 256 -> 256 -> 12, GELU (erf form) after every
hidden layer, linear output.  Loss per sample: for each slot k, the logistic loss of the
existence logit against y_k in [0, 1], plus y_k times half the squared error of the five
regression outputs.  Mean over the batch.

Everything here is plain numpy in float64, layer by layer, with no fusion; weights are taken
as given (the GPU keeps FP32 master weights and multiplies with their BF16 rounding: pass
``bf16_round(W)`` to compare).  Only the test suite imports this module.

Parity: pinned by central finite differences of the loss for every layer's weights and
biases, GELU identities (odd part, Phi(1) and its derivative), the loss at known points, the
first Adam step (-lr sign(g)) and BF16 rounding of hand-made bit patterns
(tests/test_mlp_oracle_pins.py).
"""
from __future__ import annotations

import math

import numpy as np

DIMS = (3, 256, 256, 256, 256, 12)
N_SLOT, N_REG = 2, 5


def bf16_round(x):
    """Round float32 values to bfloat16 (round to nearest, ties to even), returned as float64."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _erf(x):
    from scipy.special import erf

    return erf(x)


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(W, b, X):
    """Returns (outputs, cache).  W[l]: (in, out), b[l]: (out,), X: (B, 3)."""
    h = np.asarray(X, dtype=np.float64)
    zs, hs = [], [h]
    for l in range(len(W)):
        z = h @ W[l] + b[l]
        if l < len(W) - 1:
            zs.append(z)
            h = gelu(z)
            hs.append(h)
        else:
            out = z
    return out, (zs, hs)


def loss_and_grad_out(out, y, t):
    """Loss and dL/d(out).  y: (B, 2) existence targets in [0, 1] (1 or 0, or 0.5 where the
    pair has more solutions than slots); t: (B, 2, 5) regression targets."""
    B = out.shape[0]
    o = out.reshape(B, N_SLOT, 1 + N_REG)
    logit, reg = o[:, :, 0], o[:, :, 1:]
    # logistic loss: softplus(logit) - y logit, computed stably
    sp = np.maximum(logit, 0.0) + np.log1p(np.exp(-np.abs(logit)))
    bce = sp - y * logit
    diff = reg - t
    sq = 0.5 * y[:, :, None] * diff * diff
    L = (bce.sum() + sq.sum()) / B
    g = np.zeros_like(o)
    g[:, :, 0] = (1.0 / (1.0 + np.exp(-logit)) - y) / B
    g[:, :, 1:] = y[:, :, None] * diff / B
    return L, g.reshape(B, -1)


def backward(W, cache, g_out):
    """Gradients (dW, db) of the loss for the cache of ``forward``."""
    zs, hs = cache
    n = len(W)
    dW, db = [None] * n, [None] * n
    g = g_out
    for l in range(n - 1, -1, -1):
        dW[l] = hs[l].T @ g
        db[l] = g.sum(axis=0)
        if l > 0:
            g = (g @ W[l].T) * gelu_grad(zs[l - 1])
    return dW, db


def loss(W, b, X, y, t):
    out, _ = forward(W, b, X)
    return loss_and_grad_out(out, y, t)[0]


def grads(W, b, X, y, t):
    out, cache = forward(W, b, X)
    L, g = loss_and_grad_out(out, y, t)
    dW, db = backward(W, cache, g)
    return L, dW, db


def adam(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected); returns new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1**step)
    vh = v / (1.0 - beta2**step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
