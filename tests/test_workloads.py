"""The seeded synthetic inputs follow the recipes they state: ranges and distributions of the
ray sources and directions, the receiver lattice, the source-receiver pairs, the random
refractivity field's standard deviation and Gaussian correlation, the grid's geometry and
profile, the network's initial weights; the same seed gives the same arrays."""
import math

import numpy as np
import pytest
from scipy import stats

from paper_1810_01780_gb300 import workloads as W


def test_isotropic_sources_recipe():
    n = 200_000
    pos, d, a = W.isotropic_sources(n, 2)
    assert pos.shape == (3, n) and d.shape == (3, n) and np.all(a == 1.0)
    assert np.all(np.abs(pos[:2]) <= 400.0) and np.all((pos[2] >= 50.0) & (pos[2] <= 1500.0))
    for x, lo, hi in ((pos[0], -400, 400), (pos[1], -400, 400), (pos[2], 50, 1500)):
        assert stats.kstest(x, "uniform", args=(lo, hi - lo)).pvalue > 1e-3
    assert np.allclose(np.linalg.norm(d, axis=0), 1.0, rtol=0, atol=1e-12)
    # uniform on the sphere: cos(theta) ~ U[-1, 1], azimuth ~ U[0, 2 pi)
    assert stats.kstest(d[2], "uniform", args=(-1.0, 2.0)).pvalue > 1e-3
    phi = np.mod(np.arctan2(d[1], d[0]), 2 * math.pi)
    assert stats.kstest(phi, "uniform", args=(0.0, 2 * math.pi)).pvalue > 1e-3
    again = W.isotropic_sources(n, 2)
    assert np.array_equal(again[0], pos) and np.array_equal(again[1], d)
    assert not np.array_equal(W.isotropic_sources(n, 3)[0], pos)


def test_batched_workload_and_receivers():
    cfg = W.batched(4096)
    assert cfg["rays"][0].shape == (3, 4096)
    p = cfg["params"]
    assert (p["max_path"], p["min_amp"], p["max_generation"], p["tol"]) == (3000.0, 0.05, 3,
                                                                          1e-6)
    lay = cfg["medium"]["layers"]
    assert len(lay) == 3 and lay[0]["absorb"] and lay[2]["z_top"] == 100.0
    assert lay[2]["off"] == 0.02 and lay[1]["off"] == 0.0
    c, r = cfg["receivers"]
    assert c.shape == (64, 3) and np.all(r == 1.0)
    assert sorted(set(c[:, 0])) == sorted(set(c[:, 1])) == [-300.0, -100.0, 100.0, 300.0]
    assert sorted(set(c[:, 2])) == [25.0, 75.0, 125.0, 175.0]
    assert len({tuple(x) for x in c}) == 64


def test_point_sources_share_their_source():
    pos, d, _ = W.point_sources(4, 1000, 103)
    src = pos[:, ::1000]
    assert np.array_equal(pos, np.repeat(src, 1000, axis=1))
    assert np.all(np.abs(src[:2]) <= 200.0) and np.all((src[2] >= 100) & (src[2] <= 1500))
    assert np.allclose(np.linalg.norm(d, axis=0), 1.0, rtol=0, atol=1e-12)


def test_fan_is_an_inclusive_linspace():
    pos, d, _ = W.fan_xz(7, 240.0)
    assert np.all(pos[2] == 240.0) and np.all(pos[:2] == 0.0) and np.all(d[1] == 0.0)
    th = np.degrees(np.arctan2(d[0], d[2]))
    assert np.allclose(th, np.linspace(0.0, 180.0, 7), atol=1e-12)


def test_pairs_recipe():
    P = W.pairs(200_000, 4)
    for k, (lo, hi) in (("zs", (0, 2000)), ("zr", (0, 200)), ("dist", (0, 4000))):
        assert np.all((P[k] >= lo) & (P[k] <= hi))
        assert stats.kstest(P[k], "uniform", args=(lo, hi - lo)).pvalue > 1e-3
    na = P["n_angles"]
    assert na.dtype == np.int32 and na.min() == 32 and na.max() == 512
    assert abs(na.mean() - 272.0) < 1.0
    cfg = W.surrogate(n_train=1000, n_query=1000)
    assert not np.array_equal(cfg["train"]["zs"], cfg["queries"]["zs"])


def test_random_field_recipe():
    """Sample standard deviation sigma; autocorrelation exp(-r^2 / (2 l^2)) along each axis
    (the circular autocorrelation of the periodic field, averaged over the three axes)."""
    f = W.gaussian_random_field((64, 64, 64), 4.0, 1e-3, 20.0, 3).astype(np.float64)
    assert f.std() == pytest.approx(1e-3, rel=1e-5)
    g = f - f.mean()
    F = np.fft.rfftn(g, axes=(0, 1, 2))
    ac = np.fft.irfftn(np.abs(F) ** 2, s=g.shape, axes=(0, 1, 2))
    ac /= ac[0, 0, 0]
    for lag in (1, 2, 3, 5, 8):
        r = 4.0 * lag
        got = (ac[lag, 0, 0] + ac[0, lag, 0] + ac[0, 0, lag]) / 3.0
        assert abs(got - math.exp(-r * r / (2 * 20.0**2))) < 0.05, (lag, got)
    assert not np.array_equal(W.gaussian_random_field((16, 16, 16), 4.0, 1e-3, 20.0, 4),
                              W.gaussian_random_field((16, 16, 16), 4.0, 1e-3, 20.0, 3))


def test_grid_geometry_and_profile():
    g = W.grid_medium(8, 6, 10, spacing=4.0, sigma=0.0)
    assert g["n"].shape == (10, 6, 8) and g["n"].dtype == np.float32
    assert g["origin"] == (-14.0, -10.0, 0.0) and g["spacing"] == 4.0
    z = 4.0 * np.arange(10)
    want = (W.ICE["n0"] - W.ICE["dn"] * np.exp(-z / W.ICE["z0"])).astype(np.float32)
    assert np.array_equal(g["n"][:, 2, 3], want)
    full = W.grid_medium(8, 6, 10, spacing=4.0, sigma=1e-3, seed=3)
    dn = full["n"].astype(np.float64) - g["n"]
    assert dn.std() == pytest.approx(1e-3, rel=1e-3)


def test_network_initial_weights():
    Wt, b = W.mlp_init(0)
    assert [w.shape for w in Wt] == [(3, 256), (256, 256), (256, 256), (256, 256), (256, 12)]
    for i, w in enumerate(Wt):
        lim = math.sqrt(6.0 / w.shape[0]) if i < 4 else math.sqrt(1.0 / w.shape[0])
        assert np.abs(w).max() <= lim and np.abs(w).max() > 0.95 * lim
    assert all(np.all(c == 0.0) for c in b)
    flat = W.mlp_flatten(Wt, b)
    assert flat.size == 201_484
    W2, b2 = W.mlp_unflatten(flat)
    assert all(np.array_equal(x, y) for x, y in zip(W2, Wt))
    assert all(np.array_equal(x, y) for x, y in zip(b2, b))
