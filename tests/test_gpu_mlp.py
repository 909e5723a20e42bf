"""Surrogate network kernels (forward, loss, gradient, Adam training) vs the FP64 oracle.

The GPU multiplies BF16-rounded weights and BF16-rounded activations with FP32 accumulation;
the oracle evaluates the same BF16-rounded weights in float64 with unrounded activations.  The
tolerance follows from BF16's unit roundoff (2^-8 relative per rounded operand) accumulated over
five layers: outputs within 3e-2 relative (with an absolute floor of 3e-2 of the output
scale), the loss within 2e-2 relative, each layer's weight gradient within 5e-2 relative in
norm and at cosine similarity >= 0.998."""
import numpy as np
import pytest

from oracle import mlp
from paper_1810_01780_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rp():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1810_01780_gb300 import build

    build.build()
    import paper_1810_01780_gb300 as rp

    return rp


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
    y = rng.choice(np.array([0.0, 0.5, 1.0], np.float32), size=(n, 2), p=[0.4, 0.1, 0.5])
    t = rng.normal(0, 0.5, (n, 10)).astype(np.float32)
    return X, y, t


def _oracle_params(flat):
    Ws, bs = W.mlp_unflatten(flat)
    return [mlp.bf16_round(w) for w in Ws], [b.astype(np.float64) for b in bs]


def test_forward_matches_oracle(rp):
    net = rp.Surrogate(seed=1)
    X, _, _ = _batch(1000, 2)
    got = net.forward(X).cpu().numpy()
    Wo, bo = _oracle_params(net.get_params())
    ref, _ = mlp.forward(Wo, bo, X.astype(np.float64))
    scale = np.abs(ref).max()
    assert np.all(np.abs(got - ref) <= 3e-2 * np.abs(ref) + 3e-2 * scale)
    assert np.median(np.abs(got - ref)) <= 5e-3 * scale


def test_loss_and_gradients_match_oracle(rp):
    net = rp.Surrogate(seed=3)
    X, y, t = _batch(2048, 4)
    L, g = net.loss_grad(X, y, t)
    g = g.cpu().numpy()
    Wo, bo = _oracle_params(net.get_params())
    Lr, dW, db = mlp.grads(Wo, bo, X.astype(np.float64), y.astype(np.float64),
                           t.astype(np.float64).reshape(-1, 2, 5))
    assert abs(L - Lr) <= 2e-2 * abs(Lr)
    gW, gb = W.mlp_unflatten(g)
    for l in range(5):
        a, b = gW[l].ravel().astype(np.float64), dW[l].ravel()
        assert np.linalg.norm(a - b) <= 5e-2 * np.linalg.norm(b), l
        assert a @ b / (np.linalg.norm(a) * np.linalg.norm(b)) >= 0.998, l
        a, b = gb[l].astype(np.float64), db[l]
        assert np.linalg.norm(a - b) <= 5e-2 * np.linalg.norm(b) + 1e-6, l


def test_adam_step_matches_oracle_and_training_learns(rp):
    import torch

    net = rp.Surrogate(seed=5)
    X, y, t = _batch(4096, 6)
    p0 = net.get_params()
    xd, yd, td = (torch.as_tensor(a, device="cuda") for a in (X, y, t))
    _, g = net.loss_grad(X, y, t)
    net.train_step(xd, yd, td, 1e-3)
    p1 = net.get_params()
    # first Adam step: p1 = p0 - lr * g / (|g| + eps) elementwise (bias-corrected moments)
    g = g.cpu().numpy().astype(np.float64)
    want = p0 - 1e-3 * g / (np.abs(g) + 1e-8)
    assert np.max(np.abs(p1 - want)) <= 1e-6 + 1e-3 * 1e-3
    # a smooth target the network can fit: the loss must fall several-fold
    rng = np.random.default_rng(7)
    Xs = rng.uniform(-1, 1, (8192, 3)).astype(np.float32)
    ys = (Xs[:, :2] > 0).astype(np.float32)
    ts = np.concatenate([np.sin(2 * Xs), np.cos(Xs), np.tanh(Xs[:, :2] * Xs[:, 2:]),
                         Xs[:, :2] ** 2], axis=1)[:, :10].astype(np.float32)
    xd, yd, td = (torch.as_tensor(a, device="cuda") for a in (Xs, ys, ts))
    losses = [net.train_step(xd, yd, td, 1e-3) for _ in range(300)]
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])
