"""Pins of the FP64 surrogate-network oracle: finite differences, GELU identities, the loss
at known points, one Adam step, BF16 rounding."""
import math

import numpy as np
import pytest

from oracle import mlp
from paper_1810_01780_gb300 import workloads as W


def _small(seed=1):
    dims = (3, 8, 8, 8, 8, 12)
    Ws, bs = W.mlp_init(seed, dims)
    rng = np.random.default_rng(seed)
    Ws = [w.astype(np.float64) for w in Ws]
    bs = [rng.normal(0, 0.1, c.shape) for c in bs]
    X = rng.uniform(-1, 1, (5, 3))
    y = rng.choice([0.0, 0.5, 1.0], size=(5, 2))  # 0.5: the label of an ambiguous pair
    t = rng.normal(0, 1, (5, 2, 5))
    return Ws, bs, X, y, t


def test_gradients_match_finite_differences():
    Ws, bs, X, y, t = _small()
    L, dW, db = mlp.grads(Ws, bs, X, y, t)
    rng = np.random.default_rng(3)
    for l in range(len(Ws)):
        for _ in range(4):
            i, j = rng.integers(Ws[l].shape[0]), rng.integers(Ws[l].shape[1])
            eps = 1e-6
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[l][i, j] += eps
            Wm[l][i, j] -= eps
            fd = (mlp.loss(Wp, bs, X, y, t) - mlp.loss(Wm, bs, X, y, t)) / (2 * eps)
            assert abs(fd - dW[l][i, j]) <= 1e-7 * (1 + abs(fd)), (l, i, j)
        k = rng.integers(bs[l].shape[0])
        bp = [c.copy() for c in bs]
        bm = [c.copy() for c in bs]
        bp[l][k] += 1e-6
        bm[l][k] -= 1e-6
        fd = (mlp.loss(Ws, bp, X, y, t) - mlp.loss(Ws, bm, X, y, t)) / 2e-6
        assert abs(fd - db[l][k]) <= 1e-7 * (1 + abs(fd))


def test_gelu_identities():
    x = np.linspace(-6, 6, 241)
    assert np.allclose(mlp.gelu(x) - mlp.gelu(-x), x, atol=1e-15)  # x Phi(x) + x Phi(-x) = x
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    fd = (mlp.gelu(x + 1e-6) - mlp.gelu(x - 1e-6)) / 2e-6
    assert np.allclose(fd, mlp.gelu_grad(x), atol=1e-8)
    assert abs(mlp.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15  # Phi(1)


def test_loss_at_known_points():
    B = 4
    out = np.zeros((B, 12))
    y = np.ones((B, 2))
    t = np.zeros((B, 2, 5))
    L, _ = mlp.loss_and_grad_out(out, y, t)
    assert abs(L - 2 * math.log(2.0)) < 1e-15  # logit 0: log 2 per slot
    out[:, 0] = out[:, 6] = 40.0
    t[:] = 0.0
    L, g = mlp.loss_and_grad_out(out, y, t)
    assert L < 1e-16 and np.abs(g).max() < 1e-17
    out[:, 1] = 2.0  # one regression error of 2 in slot 0
    L, g = mlp.loss_and_grad_out(out, y, t)
    assert abs(L - 2.0) < 1e-12 and abs(g[0, 1] - 2.0 / B) < 1e-15
    L0, _ = mlp.loss_and_grad_out(out, np.zeros((B, 2)), t)  # absent: regression masked out
    assert abs(L0 - 2 * (40.0 + math.log1p(math.exp(-40.0)))) < 1e-9


def test_adam_first_step_is_signed_lr():
    g = np.array([3.0, -0.5, 1e-3])
    p, m, v = mlp.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 1e-2)
    assert np.allclose(p, -1e-2 * np.sign(g), rtol=1e-4)


def test_bf16_round():
    v = np.array([1.0, 1.0 + 2**-8, 1.0 + 3 * 2**-9, -2.5, 3.0e-3], dtype=np.float32)
    r = mlp.bf16_round(v)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2**-7 and r[3] == -2.5
    assert abs(r[4] - 3.0e-3) <= 2**-8 * 3.0e-3  # unit roundoff of 8 significant bits
