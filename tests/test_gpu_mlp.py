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


@pytest.mark.parametrize("n", [1, 1000, 70_001])
def test_gradients_match_oracle_at_ragged_sizes(rp, n):
    """Row counts that leave partial tiles (128 rows), partial weight-gradient chunks (128 rows,
    several per CTA at 70,001) and partial thin-layer chunks (64 rows)."""
    net = rp.Surrogate(seed=17)
    X, y, t = _batch(n, 18)
    L, g = net.loss_grad(X, y, t)
    g = g.cpu().numpy()
    Wo, bo = _oracle_params(net.get_params())
    Lr, dW, db = mlp.grads(Wo, bo, X.astype(np.float64), y.astype(np.float64),
                           t.astype(np.float64).reshape(-1, 2, 5))
    assert abs(L - Lr) <= 2e-2 * abs(Lr)
    gW, gb = W.mlp_unflatten(g)
    for l in range(5):
        a, b = gW[l].ravel().astype(np.float64), dW[l].ravel()
        assert np.linalg.norm(a - b) <= 5e-2 * np.linalg.norm(b) + 1e-9, l
        if n > 1:
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
    # first Adam step: p1 = p0 - lr * g / (|g| + eps) elementwise (bias-corrected moments m = g,
    # v = g^2), so no parameter moves by more than lr.  The gradient is summed with atomics in
    # no fixed order, so train_step's own evaluation differs from g in the last bits; where |g|
    # is near eps that changes g / (|g| + eps), so the formula is checked where |g| >= 1e-6 and
    # the bound everywhere.
    g = g.cpu().numpy().astype(np.float64)
    want = p0 - 1e-3 * g / (np.abs(g) + 1e-8)
    big = np.abs(g) >= 1e-6
    assert big.mean() > 0.5
    assert np.max(np.abs(p1 - want)[big]) <= 1e-6 + 1e-3 * 1e-3
    assert np.max(np.abs(p1.astype(np.float64) - p0)) <= 1e-3 * (1 + 1e-6) + 1e-7
    # a smooth target the network can fit: the loss must fall several-fold
    rng = np.random.default_rng(7)
    Xs = rng.uniform(-1, 1, (8192, 3)).astype(np.float32)
    ys = (Xs[:, :2] > 0).astype(np.float32)
    ts = np.concatenate([np.sin(2 * Xs), np.cos(Xs), np.tanh(Xs[:, :2] * Xs[:, 2:]),
                         Xs[:, :2] ** 2], axis=1)[:, :10].astype(np.float32)
    xd, yd, td = (torch.as_tensor(a, device="cuda") for a in (Xs, ys, ts))
    losses = [net.train_step(xd, yd, td, 1e-3) for _ in range(300)]
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])


def _oracle_forward_bf16_acts(Wo, bo, X):
    """The oracle's layers with every layer input rounded to BF16, as the tensor cores take it."""
    h = mlp.bf16_round(X.astype(np.float32))
    for l in range(len(Wo)):
        z = h @ Wo[l] + bo[l]
        if l == len(Wo) - 1:
            return z
        h = mlp.bf16_round(mlp.gelu(z).astype(np.float32))


@pytest.mark.parametrize("n", [1, 127, 129, 1000, 300_000])
def test_fused_inference_matches_oracle_with_bf16_activations(rp, n):
    """rp_surrogate_forward runs the fused tcgen05 kernel: one tile of 128 rows per CTA pass,
    ragged last tile; against the oracle's layers with BF16-rounded layer inputs."""
    net = rp.Surrogate(seed=11)
    X, _, _ = _batch(n, 12)
    got = net.forward(X).cpu().numpy()
    assert got.shape == (n, 12) and np.isfinite(got).all()
    Wo, bo = _oracle_params(net.get_params())
    rows = np.arange(n) if n <= 1000 else np.random.default_rng(0).choice(n, 2000, replace=False)
    ref = _oracle_forward_bf16_acts(Wo, bo, X[rows].astype(np.float64))
    scale = np.abs(ref).max()
    # FP32 accumulation in a different order may flip a BF16 rounding of an activation
    assert np.max(np.abs(got[rows] - ref)) <= 2e-2 * scale
    assert np.median(np.abs(got[rows] - ref)) <= 1e-3 * scale


def test_fused_inference_agrees_with_training_forward(rp):
    """The loss of the fused kernel's outputs (computed by the oracle's loss) equals the loss
    that the training path's own forward pass (its per-layer kernels) reports."""
    import torch

    net = rp.Surrogate(seed=13)
    X, y, t = _batch(4096, 14)
    net.train(torch.as_tensor(X, device="cuda"), torch.as_tensor(y, device="cuda"),
              torch.as_tensor(t, device="cuda"), epochs=2, batch=1024, lr=1e-3, seed=1)
    out = net.forward(X).cpu().numpy().astype(np.float64)
    L_fused, _ = mlp.loss_and_grad_out(out, y.astype(np.float64), t.astype(np.float64).reshape(-1, 2, 5))
    L_train, _ = net.loss_grad(X, y, t)
    assert abs(L_fused - L_train) <= 2e-3 * abs(L_train), (L_fused, L_train)


def test_a_wait_that_runs_out_returns_an_error_and_leaves_the_context_usable(rp):
    """The tensor-core kernels bound every wait for their own bulk copies and matrix products.
    With the bound set to one SM cycle the first wait gives up before the 128 KB weight copy can
    land: the CTA records it, drains the work it issued (with the default bound), frees its
    tensor memory and returns, and the call returns RP_ERR_TIMEOUT -- no trap, no hang.  With
    the default bound back, the same calls give the results of a fresh network."""
    import numpy as np

    from paper_1810_01780_gb300 import _abi as A

    net = rp.Surrogate(seed=3)
    X = np.random.default_rng(1).uniform(-1, 1, (4096, 3)).astype(np.float32)
    y = np.zeros((4096, 2), np.float32)
    t = np.zeros((4096, 10), np.float32)
    ref = net.forward(X).cpu().numpy()
    ref_loss, _ = net.loss_grad(X, y, t)
    net.set_wait_limit(1)
    with pytest.raises(A.RPError) as e:
        net.forward(X)
    assert e.value.code == -6 and "gave up" in str(e.value)
    with pytest.raises(A.RPError) as e:
        net.loss_grad(X, y, t)
    assert e.value.code == -6
    net.set_wait_limit(0)
    np.testing.assert_array_equal(net.forward(X).cpu().numpy(), ref)
    loss, _ = net.loss_grad(X, y, t)
    assert abs(loss - ref_loss) <= 1e-9 * abs(ref_loss)
    with pytest.raises(A.RPError):
        net.set_wait_limit(-1)
