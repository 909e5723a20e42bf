"""Pins of the oracle's non-horizontal boundaries (boundary shapes beyond the plane, Sec. 2, the
paragraph after Fig. 1): tilted planes and height-field surfaces between layers.

Each check is exact geometry written out here, independent of the oracle's code path:
- straight rays in constant layers meeting a tilted plane: intersection point (ray-plane
  intersection), mirror reflection about the plane's normal, vector Snell refraction,
  Fresnel amplitudes, travel times; total internal reflection past the critical angle;
- a height field sampled from a plane reproduces that plane's rays (the bilinear interpolant of
  a linear function is the function);
- a saddle cell z = z0 + h u v (one raised corner): a vertical ray's landing depth and its
  reflection off the saddle's local normal, from the saddle's own closed form;
- around a rough height field between exponential profiles every ray, primaries and
  secondaries, ends on its own side of the surface;
- the start layer of points above, on and below a tilted plane and a height field."""
import math

import numpy as np
import pytest

import oracle
from oracle.analytic import C0
from paper_1810_01780_gb300 import workloads as W


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def _two_constant_layers(n_top, n_bot, normal, z0=100.0, absorb_top=False, height=None):
    srf = dict(layer=1, normal=tuple(normal))
    if height is not None:
        srf.update(height)
    return {"kind": "layered", "layers": [dict(n0=n_top, absorb=absorb_top),
                                          dict(z_top=z0, n0=n_bot)], "surfaces": [srf]}


def _fresnel_s(n1, n2, ci, ct):
    return (n1 * ci - n2 * ct) / (n1 * ci + n2 * ct), 2 * n1 * ci / (n1 * ci + n2 * ct)


def test_tilted_plane_exact_geometry(oracle_lib):
    """Rays from below a tilted plane (normal N, through (0, 0, 100 m)) in constant layers
    n = 1.5 below and 1.0 above: the primary reflects about N at the ray-plane intersection,
    the secondary leaves along the vector Snell direction; end points after 400 m of path,
    travel times and s-polarised amplitudes are exact; past the critical angle there is no
    secondary and |r| = 1."""
    N = _unit([0.25, -0.15, 1.0])
    n1, n2, z0, S = 1.5, 1.0, 100.0, 400.0
    med = _two_constant_layers(n2, n1, N, z0)
    dirs = [_unit(v) for v in ([0.3, 0.1, -1.0], [-0.2, 0.4, -1.0], [0.05, 0.0, -1.0],
                               [1.0, 0.2, -0.6], [-0.9, -0.3, -0.35])]
    p0 = np.array([10.0, 20.0, 180.0])
    pos = np.repeat(p0[:, None], len(dirs), axis=1)
    d = np.stack(dirs, axis=1)
    prm = dict(W.TRACE_DEFAULTS, max_path=S)
    rays, _ = oracle.trace(med, prm, pos, d)
    P0 = np.array([0.0, 0.0, z0])
    n_tir = 0
    for i, t in enumerate(dirs):
        lam = N @ (P0 - p0) / (N @ t)  # the plane N . (r - P0) = 0
        hit = p0 + lam * t
        ci = -(t @ N)  # N points into the incident (lower) layer
        t_r = t - 2 * (t @ N) * N
        prim = rays[i]
        assert prim["n_refl"] == 1 and prim["status"] == oracle.STATUS["MAX_PATH"]
        assert np.allclose(prim["pos"], hit + (S - lam) * t_r, atol=1e-7), i
        assert np.allclose(prim["dir"], t_r, atol=1e-12)
        assert abs(prim["time"] - n1 * S / C0) < 1e-17
        sec = rays[rays["parent"] == i]
        eta = n1 / n2
        s2 = eta * eta * (1 - ci * ci)
        if s2 > 1:
            n_tir += 1
            assert len(sec) == 0 and abs(prim["amp"] - 1.0) < 1e-15
            continue
        ct = math.sqrt(1 - s2)
        t_t = eta * t + (eta * ci - ct) * N
        rs, ts = _fresnel_s(n1, n2, ci, ct)
        assert abs(prim["amp"] - rs) < 1e-12
        assert len(sec) == 1
        s = sec[0]
        assert s["gen"] == 1 and s["layer"] == 0 and s["status"] == oracle.STATUS["MAX_PATH"]
        assert abs(s["amp"] - ts) < 1e-12
        assert np.allclose(s["dir"], t_t, atol=1e-12)
        assert np.allclose(s["pos"], hit + (S - lam) * t_t, atol=1e-7), i
        assert abs(s["time"] - (n1 * lam + n2 * (S - lam)) / C0) < 1e-17
    assert 0 < n_tir < len(dirs)
    # from above (n = 1.0 onto n = 1.5): the normal toward the incident side is -N
    up = [_unit(v) for v in ([0.2, -0.1, 1.0], [-0.6, 0.3, 1.0])]
    p1 = np.array([-15.0, 5.0, 40.0])
    rays, _ = oracle.trace(med, prm, np.repeat(p1[:, None], len(up), axis=1),
                           np.stack(up, axis=1))
    for i, t in enumerate(up):
        lam = N @ (P0 - p1) / (N @ t)
        hit = p1 + lam * t
        Ni = -N
        ci = -(t @ Ni)
        eta = n2 / n1
        ct = math.sqrt(1 - eta * eta * (1 - ci * ci))
        t_t = eta * t + (eta * ci - ct) * Ni
        t_r = t - 2 * (t @ N) * N
        rs, ts = _fresnel_s(n2, n1, ci, ct)
        prim, sec = rays[i], rays[rays["parent"] == i]
        assert np.allclose(prim["pos"], hit + (S - lam) * t_r, atol=1e-7)
        assert abs(prim["amp"] - rs) < 1e-12 and len(sec) == 1 and sec[0]["layer"] == 1
        assert np.allclose(sec[0]["pos"], hit + (S - lam) * t_t, atol=1e-7)
        assert abs(sec[0]["amp"] - ts) < 1e-12


def _plane_heights(a, b, nx=81, ny=61, ox=-400.0, oy=-300.0, dx=10.0, dy=10.0):
    x = ox + dx * np.arange(nx)
    y = oy + dy * np.arange(ny)
    return dict(height=a * x[None, :] + b * y[:, None], origin=(ox, oy), spacing=(dx, dy))


def test_height_field_of_a_plane_reproduces_the_tilted_plane(oracle_lib):
    """The heights of the plane z = z0 + a x + b y on a node grid (and a flat base plane) give,
    inside the grid, the same surface as the tilted plane of normal (-a, -b, 1): every ray record
    of a workload with refraction into an exponential profile agrees to rounding."""
    a, b = 0.12, -0.07
    N = _unit([-a, -b, 1.0])
    layers = [dict(n0=1.0003, absorb=False),
              dict(z_top=60.0, n0=1.78, dn=0.46, z0=75.0, off=0.0)]
    tilted = {"kind": "layered", "layers": layers, "surfaces": [dict(layer=1, normal=tuple(N))]}
    hf = {"kind": "layered", "layers": layers,
          "surfaces": [dict(layer=1, normal=(0.0, 0.0, 1.0), **_plane_heights(a, b))]}
    rng = np.random.default_rng(4)
    n = 64
    pos = np.stack([rng.uniform(-60, 60, n), rng.uniform(-50, 50, n), rng.uniform(70, 140, n)])
    d = W.isotropic_dirs(rng, n)
    d[2] = -np.abs(d[2])  # upward, toward the surface
    prm = dict(W.TRACE_DEFAULTS, max_path=150.0)
    r1, _ = oracle.trace(tilted, prm, pos, d)
    r2, _ = oracle.trace(hf, prm, pos, d)
    assert len(r1) == len(r2) and (r1["n_refl"] > 0).sum() > 20 and (r1["parent"] >= 0).any()
    for k in ("status", "layer", "n_acc", "n_refl", "parent", "seq"):
        np.testing.assert_array_equal(r1[k], r2[k], err_msg=k)
    for k, tol in (("pos", 1e-9), ("dir", 1e-11), ("path", 1e-9), ("time", 1e-17),
                   ("amp", 1e-12)):
        assert np.abs(r1[k] - r2[k]).max() <= tol, k


def test_height_field_saddle_landing_and_local_normal(oracle_lib):
    """One raised corner of a cell gives the saddle z = z0 + h u v (u, v the cell's fractional
    coordinates): a vertical ray from below at (u, v) lands at that depth and reflects about
    the saddle's normal (-h v / dx, -h u / dy, 1) / |...|, exact geometry in constant media."""
    z0, h, dx, dy = 100.0, 4.0, 10.0, 8.0
    heights = np.zeros((3, 3))
    heights[2, 2] = h  # node (i, j) = (2, 2) at (dx, dy): the far corner of the cell [0, dx] x [0, dy]
    srf = dict(height=heights, origin=(-dx, -dy), spacing=(dx, dy))
    med = _two_constant_layers(1.0, 1.5, (0.0, 0.0, 1.0), z0, height=srf)
    uv = [(0.5, 0.5), (0.2, 0.9), (0.75, 0.3)]
    pos = np.array([[u * dx for u, v in uv], [v * dy for u, v in uv], [150.0] * len(uv)])
    d = np.tile(np.array([[0.0], [0.0], [-1.0]]), (1, len(uv)))
    S = 80.0
    rays, _ = oracle.trace(med, dict(W.TRACE_DEFAULTS, max_path=S), pos, d)
    for i, (u, v) in enumerate(uv):
        zb = z0 + h * u * v
        N = _unit([-h * v / dx, -h * u / dy, 1.0])
        t = np.array([0.0, 0.0, -1.0])
        t_r = t - 2 * (t @ N) * N
        hit = np.array([u * dx, v * dy, zb])
        prim = rays[i]
        assert prim["n_refl"] == 1
        assert np.allclose(prim["dir"], t_r, atol=1e-12)
        assert np.allclose(prim["pos"], hit + (S - (150.0 - zb)) * t_r, atol=1e-7)
        z, gx, gy = oracle.OracleMedium(med).boundary_depth(1, u * dx, v * dy)
        assert abs(z - zb) < 1e-12 and abs(gx - h * v / dx) < 1e-12 and abs(gy - h * u / dy) < 1e-12


def test_every_ray_ends_on_its_own_side_of_a_rough_surface(oracle_lib):
    """Isotropic rays around a rough height field (seeded node heights, 2 m spacing) over a
    tilted base plane between exponential profiles: every ray -- primaries and the secondaries
    cast at the surface -- ends in the layer it was traced in (its end point on its own side of
    the surface, or on it), and every split's reflected direction leaves the surface (a wrong
    normal would send rays through it)."""
    rng = np.random.default_rng(12)
    ny, nx = 41, 51
    heights = rng.normal(0.0, 0.8, (ny, nx))
    srf = dict(layer=1, normal=tuple(_unit([0.05, -0.03, 1.0])), height=heights,
               origin=(-50.0, -40.0), spacing=(2.0, 2.0))
    med = {"kind": "layered", "layers": [dict(n0=1.78, dn=0.46, z0=75.0),
                                         dict(z_top=60.0, n0=1.78, dn=0.46, z0=75.0, off=0.03)],
           "surfaces": [srf]}
    m = oracle.OracleMedium(med)
    n = 400
    pos = np.stack([rng.uniform(-40, 40, n), rng.uniform(-30, 30, n), rng.uniform(45, 75, n)])
    d = W.isotropic_dirs(rng, n)
    prm = dict(W.TRACE_DEFAULTS, max_path=60.0, max_generation=2)
    rays, _ = oracle.trace(med, prm, pos, d)
    assert (rays["n_refl"] > 0).sum() > 50 and (rays["gen"] == 2).any()
    # a reflected ray leaves the surface: within 60 m of path it meets the rough surface again
    # only a few times, and the secondaries stay few (a normal turned the wrong way lets rays
    # creep along the surface, splitting at every step)
    assert len(rays) < 3 * n and rays["n_refl"].max() <= 10
    for r in rays:
        z, _, _ = m.boundary_depth(1, r["pos"][0], r["pos"][1])
        side = r["pos"][2] - z
        assert (side >= -1e-9) if r["layer"] == 1 else (side <= 1e-9), (r["layer"], side)


def test_start_layer_at_tilted_plane_and_height_field(oracle_lib):
    N = _unit([0.3, 0.0, 1.0])
    m = oracle.OracleMedium(_two_constant_layers(1.0, 1.5, N, 100.0))
    # the plane z = 100 - 0.3 x
    assert m.layer_at(np.array([100.0, 0.0, 70.0 + 1e-9])) == 1
    assert m.layer_at(np.array([100.0, 0.0, 70.0])) == 1  # on the boundary: the layer below
    assert m.layer_at(np.array([100.0, 0.0, 70.0 - 1e-9])) == 0
    assert m.layer_at(np.array([-100.0, 0.0, 120.0])) == 0
    hf = oracle.OracleMedium(_two_constant_layers(
        1.0, 1.5, (0.0, 0.0, 1.0), 100.0, height=_plane_heights(0.0, 0.5)))
    assert hf.layer_at(np.array([0.0, 20.0, 109.0])) == 0
    assert hf.layer_at(np.array([0.0, 20.0, 111.0])) == 1
    # beyond the nodes the field is held at its edge value (y = 300: 150 m)
    assert hf.layer_at(np.array([0.0, 500.0, 249.0])) == 0
    assert hf.layer_at(np.array([0.0, 500.0, 251.0])) == 1
