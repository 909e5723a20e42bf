"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own code path: Runge-Kutta order conditions,
closed-form ray solutions of the exponential profile, exact straight-line geometry at
constant n, Fresnel energy conservation, brute-force step refinement, the accuracy class the
paper prints (Sec. 2, accuracy study; tests/golden/paper_accuracy.json).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle.analytic import C0, ExpProfile, solutions
from paper_1810_01780_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------------------
# Cash-Karp tableau
# --------------------------------------------------------------------------------------

def _conditions(A, b, c):
    Ac = A @ c
    return {
        (1, "b"): (b.sum(), 1.0),
        (2, "bc"): (b @ c, 1 / 2),
        (3, "bc2"): (b @ c**2, 1 / 3),
        (3, "bAc"): (b @ Ac, 1 / 6),
        (4, "bc3"): (b @ c**3, 1 / 4),
        (4, "bcAc"): (b @ (c * Ac), 1 / 8),
        (4, "bAc2"): (b @ (A @ c**2), 1 / 12),
        (4, "bAAc"): (b @ (A @ Ac), 1 / 24),
        (5, "bc4"): (b @ c**4, 1 / 5),
        (5, "bc2Ac"): (b @ (c**2 * Ac), 1 / 10),
        (5, "b(Ac)2"): (b @ Ac**2, 1 / 20),
        (5, "bcAc2"): (b @ (c * (A @ c**2)), 1 / 15),
        (5, "bAc3"): (b @ (A @ c**3), 1 / 20),
        (5, "bcAAc"): (b @ (c * (A @ Ac)), 1 / 30),
        (5, "bA(cAc)"): (b @ (A @ (c * Ac)), 1 / 40),
        (5, "bAAc2"): (b @ (A @ (A @ c**2)), 1 / 60),
        (5, "bAAAc"): (b @ (A @ (A @ Ac)), 1 / 120),
    }


def test_tableau_order_conditions(oracle_lib):
    c, a, b5, b4 = oracle.ck_tableau()
    A = np.zeros((6, 6))
    A[:, :5] = a
    assert np.allclose(A.sum(axis=1), c, atol=1e-15, rtol=0)  # row-sum condition
    assert np.all(np.triu(A) == 0.0)  # explicit method
    for (order, name), (got, want) in _conditions(A, b5, c).items():
        assert abs(got - want) < 1e-14, ("b5", name)
    bad = 0
    for (order, name), (got, want) in _conditions(A, b4, c).items():
        if order <= 4:
            assert abs(got - want) < 1e-14, ("b4", name)
        else:
            bad += abs(got - want) > 1e-6
    assert bad > 0  # the embedded weights are genuinely only fourth order


@pytest.mark.parametrize("k", range(7))
def test_tableau_polynomial_exactness(oracle_lib, k):
    # y' = x^k from x0 = 0.3 over h = 0.7: exact increment ((x0+h)^(k+1) - x0^(k+1)) / (k+1)
    coef = np.zeros(k + 1)
    coef[k] = 1.0
    x0, h = 0.3, 0.7
    y5, y4 = oracle.ck_poly_step(coef, x0, 0.0, h)
    exact = ((x0 + h) ** (k + 1) - x0 ** (k + 1)) / (k + 1)
    if k <= 4:
        assert abs(y5 - exact) < 1e-14
    else:
        assert abs(y5 - exact) > 1e-8
    if k <= 3:
        assert abs(y4 - exact) < 1e-14
    else:
        assert abs(y4 - exact) > 1e-8


def test_ray_step_local_order(oracle_lib):
    """One step of the ray system: error vs a 4096-substep reference scales like h^6."""
    med = oracle.OracleMedium(W.single_profile())
    th = math.radians(100.0)
    y0 = np.array([0.0, 0.0, 30.0, math.sin(th), 0.0, math.cos(th), 0.0])
    errs = []
    hs = [16.0, 8.0, 4.0]
    for h in hs:
        y1, _ = oracle.ck_step(med, y0, h)
        yr = y0.copy()
        for _ in range(4096):
            yr, _ = oracle.ck_step(med, yr, h / 4096)
        errs.append(np.linalg.norm(y1[:6] - yr[:6]))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(len(hs) - 1)]
    assert all(5.0 < s < 7.0 for s in slopes), (errs, slopes)


@pytest.mark.parametrize("theta_deg", [60.0, 100.0, 170.0])
def test_error_measure_is_per_unit_step(oracle_lib, theta_deg):
    """The step's error measure takes the position part of the embedded difference per unit
    step length (|dr| / h) beside the direction part (|dt|).  The difference of a fifth- and
    a fourth-order solution is O(h^5) in every component, so the measure falls like h^4 as h
    halves (like h^5 if the position part were not divided by h)."""
    med = oracle.OracleMedium(W.single_profile())
    th = math.radians(theta_deg)
    y0 = np.array([0.0, 0.0, 30.0, math.sin(th), 0.0, math.cos(th), 0.0])
    hs = [4.0, 2.0, 1.0, 0.5]
    es = [oracle.ck_step(med, y0, h)[1] for h in hs]
    slopes = [math.log2(es[i] / es[i + 1]) for i in range(len(hs) - 1)]
    assert all(3.8 < q < 4.2 for q in slopes), (es, slopes)


# --------------------------------------------------------------------------------------
# ray equations
# --------------------------------------------------------------------------------------

def test_rhs_projection_and_index(oracle_lib):
    med = oracle.OracleMedium(W.single_profile())
    t = np.array([0.6, 0.0, -0.8])
    y = np.array([1.0, 2.0, 40.0, *t, 0.0])
    k = oracle.rhs(med, y)
    n = 1.788 - 0.463 * math.exp(-40.0 / 75.0)
    g = 0.463 / 75.0 * math.exp(-40.0 / 75.0)
    assert np.allclose(k[:3], t, rtol=0, atol=0)
    assert abs(k[6] - n / C0) < 1e-22
    # tangent derivative is orthogonal to t and equals the transverse part of grad n / n
    assert abs(k[3:6] @ t) < 1e-18
    want = (np.array([0.0, 0.0, g]) - g * t[2] * t) / n
    assert np.allclose(k[3:6], want, rtol=1e-15, atol=0)
    kp = oracle.rhs(med, y, rhs_form="paraxial")
    assert np.allclose(kp[3:6], [0.0, 0.0, g / n], rtol=1e-15, atol=0)


def test_straight_lines_constant_index(oracle_lib):
    med = {"kind": "layered", "layers": [dict(n0=1.5, dn=0.0)]}
    rng = np.random.default_rng(11)
    n = 64
    pos = rng.uniform(-100, 100, (3, n))
    d = W.isotropic_dirs(rng, n)
    prm = dict(W.TRACE_DEFAULTS, max_path=1234.5)
    rays, _ = oracle.trace(med, prm, pos, d)
    assert np.all(rays["status"] == oracle.STATUS["MAX_PATH"])
    end = pos.T + 1234.5 * d.T
    assert np.max(np.abs(rays["pos"] - end)) < 1e-9
    assert np.max(np.abs(rays["dir"] - d.T)) < 1e-14
    assert np.max(np.abs(rays["time"] / (1.5 * 1234.5 / C0) - 1.0)) < 1e-13
    assert np.all(rays["path"] == 1234.5)
    assert np.all(rays["n_rej"] == 0)


def _fan_single_profile(tol, h_max=10.0, max_path=1500.0, depth=200.0, n=23,
                        rhs_form="projected"):
    med = W.single_profile()
    pos, d, a = W.fan_xz(n, depth, 3.0, 177.0)
    prm = dict(W.TRACE_DEFAULTS, tol=tol, h_max=h_max, h0=h_max, max_path=max_path,
               max_generation=0, rhs_form=rhs_form)
    rays, _ = oracle.trace(med, prm, pos, d, a)
    return pos, d, rays


@pytest.mark.parametrize("form", ["projected", "momentum"])
def test_snell_invariant_conserved(oracle_lib, form):
    prof = ExpProfile()
    pos, d, rays = _fan_single_profile(1e-6, rhs_form=form)
    p0 = prof.n(pos[2]) * np.hypot(d[0], d[1])
    p1 = prof.n(rays["pos"][:, 2]) * np.hypot(rays["dir"][:, 0], rays["dir"][:, 1])
    assert np.max(np.abs(p1 - p0)) < 1e-6


@pytest.mark.parametrize("form", ["projected", "momentum"])
def test_closed_form_range_path_time(oracle_lib, form):
    """End point on the closed-form curve X(z); S and T match the closed forms -- for Eq. 1
    expanded for a unit tangent (projected) and integrated as written on p = n t (momentum)."""
    prof = ExpProfile()
    pos, d, rays = _fan_single_profile(1e-9, rhs_form=form)
    th = np.arctan2(d[0], d[2])
    # the momentum form controls the error of p / n, not of t: its global error stays within
    # tol * S (1.5e-6 m here) but is not as far below it as the projected form's
    lim = 2e-7 if form == "projected" else 1e-6
    for i, r in enumerate(rays):
        X, S, T = prof.ray_to_depth(pos[2, i], th[i], r["pos"][2], ends_down=r["dir"][2] > 0)
        assert abs(r["pos"][0] - X) < lim, i
        assert abs(r["path"] - S) < lim, i
        assert abs(r["time"] - T) < 1e-15, i


def test_layer_offset_shifts_the_profile(oracle_lib):
    """A layer's index n0 - dn exp(-z/z0) + off: the profile written with n0 lowered by 0.02
    and off = +0.02 is the same medium, so its rays lie on the closed-form curves of a = n0."""
    prof = ExpProfile()
    med = {"kind": "layered", "layers": [dict(n0=prof.a - 0.02, dn=prof.b, z0=prof.zeta,
                                              off=0.02)]}
    pos, d, a = W.fan_xz(9, 200.0, 3.0, 177.0)
    prm = dict(W.TRACE_DEFAULTS, tol=1e-9, max_path=1500.0, max_generation=0)
    rays, _ = oracle.trace(med, prm, pos, d, a)
    th = np.arctan2(d[0], d[2])
    for i, r in enumerate(rays):
        X, S, T = prof.ray_to_depth(pos[2, i], th[i], r["pos"][2], ends_down=r["dir"][2] > 0)
        assert abs(r["pos"][0] - X) < 2e-7 and abs(r["time"] - T) < 1e-15, i
    # a constant layer (dn = 0) with an offset: n = n0 + off along a straight line
    med = {"kind": "layered", "layers": [dict(n0=1.3, dn=0.0, off=0.2)]}
    rays, _ = oracle.trace(med, dict(prm, max_path=100.0), pos[:, :1], d[:, :1])
    assert abs(rays[0]["time"] - 1.5 * 100.0 / C0) < 1e-18


def test_start_layer_from_depth(oracle_lib):
    """A ray starts in the layer that holds its depth: a boundary depth itself belongs to the
    layer below it.  Straight vertical rays in constant layers (n 1.3 above 100 m, 1.5
    below) started at 99.5, 100 and 100.5 m, going down 50 m: T = n s / c0 of their layer."""
    med = {"kind": "layered", "layers": [dict(n0=1.3), dict(z_top=100.0, n0=1.5)]}
    z = np.array([99.5, 100.0, 100.5])
    pos = np.stack([np.zeros(3), np.zeros(3), z])
    d = np.stack([np.zeros(3), np.zeros(3), np.ones(3)])
    prm = dict(W.TRACE_DEFAULTS, max_path=50.0, max_generation=0)
    rays, _ = oracle.trace(med, prm, pos, d)
    # the first ray crosses the boundary after 0.5 m (n_refl = 1, reflected back up); the
    # others never meet a boundary
    assert list(rays["n_refl"]) == [1, 0, 0]
    for i in (1, 2):
        assert abs(rays[i]["time"] - 1.5 * 50.0 / C0) < 1e-18
        assert rays[i]["pos"][2] == pytest.approx(z[i] + 50.0, abs=1e-9)


def test_step_growth_and_inherited_step(oracle_lib):
    """The step law at zero error (constant index): every accepted step grows the next by the
    growth limit 5, up to h_max.  From h0 = 0.01 m with h_max = 10 m the steps are 0.01,
    0.05, 0.25, 1.25, 6.25, then 10 m; 100 m of path take 5 + 10 (the last one shortened to
    the path limit) = 15 accepted steps.  A secondary starts with its parent's step at the
    split: a ray across an internal plane at 50 m depth (normal incidence, constant indices)
    has taken 0.01..6.25 (7.81 m) and four more steps of 10 m (47.81 m) before the 2.19 m
    step that lands on the plane; its next step (10 m) is the secondary's first, so the
    secondary covers the remaining 50 m in 5 steps."""
    med = {"kind": "layered", "layers": [dict(n0=1.5)]}
    prm = dict(W.TRACE_DEFAULTS, h0=0.01, h_max=10.0, max_path=100.0, max_generation=0)
    rays, _ = oracle.trace(med, prm, np.zeros((3, 1)), np.array([[0.0], [0.0], [1.0]]))
    assert rays[0]["n_acc"] == 15 and rays[0]["n_rej"] == 0
    med = {"kind": "layered", "layers": [dict(n0=1.5), dict(z_top=50.0, n0=1.6)]}
    rays, _ = oracle.trace(med, dict(prm, max_generation=1), np.zeros((3, 1)),
                           np.array([[0.0], [0.0], [1.0]]))
    sec = rays[rays["parent"] == 0]
    assert len(sec) == 1 and sec[0]["status"] == oracle.STATUS["MAX_PATH"]
    assert sec[0]["n_acc"] == 5


def test_error_shrinks_with_tolerance(oracle_lib):
    """Brute force: tol 1e-12 with h_max 0.5 m as reference; the end-point error falls with tol."""
    prof = ExpProfile()
    _, _, ref = _fan_single_profile(1e-12, h_max=0.5, n=9)
    errs = []
    for tol in (1e-4, 1e-6, 1e-8):
        _, _, r = _fan_single_profile(tol, n=9)
        errs.append(np.max(np.linalg.norm(r["pos"] - ref["pos"], axis=1)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-5
    # the reference itself sits on the closed-form curve
    pos, d, _ = W.fan_xz(9, 200.0, 3.0, 177.0)
    th = np.arctan2(d[0], d[2])
    for i, r in enumerate(ref):
        X, _, _ = prof.ray_to_depth(200.0, th[i], r["pos"][2], ends_down=r["dir"][2] > 0)
        assert abs(r["pos"][0] - X) < 1e-7


def test_paraxial_form_is_less_accurate(oracle_lib):
    """Eq. 2 taken literally (t' = grad n / n, t renormalised per step) drifts from the
    closed form far more than the projected form at the same tolerance."""
    prof = ExpProfile()
    med = W.single_profile()
    pos, d, a = W.fan_xz(5, 200.0, 60.0, 120.0)
    th = np.arctan2(d[0], d[2])
    worst = {}
    for form in ("projected", "paraxial"):
        prm = dict(W.TRACE_DEFAULTS, tol=1e-8, max_path=1500.0, max_generation=0, rhs_form=form)
        rays, _ = oracle.trace(med, prm, pos, d, a)
        e = []
        for i, r in enumerate(rays):
            X, _, _ = prof.ray_to_depth(200.0, th[i], r["pos"][2], ends_down=r["dir"][2] > 0)
            e.append(abs(r["pos"][0] - X))
        worst[form] = max(e)
    assert worst["projected"] < 1e-5
    assert worst["paraxial"] > 100 * worst["projected"]


# --------------------------------------------------------------------------------------
# boundary module
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("pol", ["s", "p", "unpol"])
def test_fresnel_energy_conservation(oracle_lib, pol):
    rng = np.random.default_rng(5)
    for _ in range(200):
        n1, n2 = rng.uniform(1.0, 2.0, 2)
        ci = rng.uniform(0.0, 1.0)
        s2 = (n1 / n2) ** 2 * (1 - ci * ci)
        if s2 > 1:
            continue
        ct = math.sqrt(1 - s2)
        r, tau = oracle.fresnel(n1, n2, ci, ct, pol)
        if pol == "unpol":
            R, T = r * r, tau * tau
        else:
            R, T = r * r, (n2 * ct) / (n1 * ci) * tau * tau if ci > 0 else 0.0
        assert abs(R + T - 1.0) < 1e-12


def test_fresnel_special_cases(oracle_lib):
    # normal incidence
    for pol in ("s", "p"):
        r, tau = oracle.fresnel(1.78, 1.0, 1.0, 1.0, pol)
        rs = (1.78 - 1.0) / (1.78 + 1.0)
        assert abs(abs(r) - rs) < 1e-15
        assert abs(tau - 2 * 1.78 / 2.78) < 1e-15
    # s: r = (n1 - n2)/(n1 + n2); p has the opposite sign convention at normal incidence
    assert oracle.fresnel(1.78, 1.0, 1.0, 1.0, "s")[0] > 0
    assert oracle.fresnel(1.78, 1.0, 1.0, 1.0, "p")[0] < 0
    # matched media: no reflection, full transmission, undeviated
    t = np.array([0.3, 0.2, -math.sqrt(1 - 0.13)])
    tr, tt, r, tau, tir = oracle.split(t, np.array([0.0, 0.0, 1.0]), 1.4, 1.4)
    assert not tir and abs(r) < 1e-15 and abs(tau - 1) < 1e-15
    assert np.allclose(tt, t, atol=1e-15)
    assert np.allclose(tr, [t[0], t[1], -t[2]], atol=1e-15)
    # Brewster angle: r_p = 0
    n1, n2 = 1.0, 1.5
    tb = math.atan(n2 / n1)
    ct = math.sqrt(1 - (n1 / n2 * math.sin(tb)) ** 2)
    assert abs(oracle.fresnel(n1, n2, math.cos(tb), ct, "p")[0]) < 1e-15


def test_snell_vector_refraction_and_tir(oracle_lib):
    rng = np.random.default_rng(8)
    nrm = np.array([0.0, 0.0, 1.0])  # toward the incident side (+z, deeper)
    for _ in range(200):
        n1, n2 = rng.uniform(1.0, 1.9, 2)
        t = W.isotropic_dirs(rng, 1)[:, 0]
        t[2] = -abs(t[2])  # moving up, against the normal
        tr, tt, r, tau, tir = oracle.split(t, nrm, n1, n2)
        sin_i = math.hypot(t[0], t[1])
        assert abs(np.linalg.norm(tr) - 1) < 1e-15
        assert np.allclose(tr, [t[0], t[1], -t[2]], atol=1e-15)
        if n1 * sin_i > n2:
            assert tir and r == 1.0 and tau == 0.0
            continue
        assert not tir
        assert abs(np.linalg.norm(tt) - 1) < 1e-15
        sin_t = math.hypot(tt[0], tt[1])
        assert abs(n1 * sin_i - n2 * sin_t) < 1e-14  # Snell's law
        assert abs(np.dot(np.cross(t, nrm), tt)) < 1e-14  # plane of incidence
        assert tt[2] < 0  # transmitted onward


def test_boundary_split_constant_layers(oracle_lib):
    """Straight rays in two constant layers: intersection, reflection, refraction and amplitudes
    are exact geometry."""
    n_air, n_ice = 1.0, 1.5
    med = {"kind": "layered", "layers": [dict(n0=n_air, absorb=True), dict(z_top=0.0, n0=n_ice)]}
    th = np.radians([120.0, 140.0, 160.0, 179.0, 135.0])  # all moving up toward z = 0
    n = len(th)
    pos = np.zeros((3, n))
    pos[2] = 50.0
    d = np.stack([np.sin(th), np.zeros(n), np.cos(th)])
    prm = dict(W.TRACE_DEFAULTS, max_path=200.0)
    rays, _ = oracle.trace(med, prm, pos, d)
    for i in range(n):
        ci = -d[2, i]
        s_hit = 50.0 / ci
        x_hit = s_hit * d[0, i]
        prim = rays[i]
        assert prim["n_refl"] == 1
        # after reflection: straight on to s = 200 with t_z flipped
        end = np.array([x_hit, 0.0, 0.0]) + (200.0 - s_hit) * np.array([d[0, i], 0.0, ci])
        assert np.allclose(prim["pos"], end, atol=1e-8)
        s2 = (n_ice / n_air) ** 2 * (1 - ci * ci)
        sec = rays[(rays["parent"] == i)]
        if s2 > 1:
            assert abs(prim["amp"] - 1.0) < 1e-15 and len(sec) == 0
            continue
        ct = math.sqrt(1 - s2)
        rs = (n_ice * ci - n_air * ct) / (n_ice * ci + n_air * ct)
        ts = 2 * n_ice * ci / (n_ice * ci + n_air * ct)
        assert abs(prim["amp"] - rs) < 1e-12
        assert len(sec) == 1
        s = sec[0]
        assert s["status"] == oracle.STATUS["TRANSMITTED"] and s["gen"] == 1
        assert s["pos"][2] == 0.0  # the landing point is put on the plane exactly
        assert abs(s["amp"] - ts) < 1e-12
        assert np.allclose(s["pos"], [x_hit, 0.0, 0.0], atol=1e-8)
        assert abs(s["path"] - s_hit) < 1e-8
        assert abs(s["time"] - n_ice * s_hit / C0) < 1e-18
        assert abs(n_ice * math.sqrt(1 - ci * ci) - n_air * math.hypot(*s["dir"][:2])) < 1e-12


def test_internal_boundary_secondary_traced(oracle_lib):
    """A traced secondary continues straight in the far layer; generation cap honoured."""
    med = {"kind": "layered",
           "layers": [dict(n0=1.3), dict(z_top=100.0, n0=1.5), dict(z_top=200.0, n0=1.3)]}
    th = math.radians(30.0)
    pos = np.array([[0.0], [0.0], [150.0]])
    d = np.array([[math.sin(th)], [0.0], [math.cos(th)]])
    for gmax in (0, 1, 3):
        prm = dict(W.TRACE_DEFAULTS, max_path=400.0, max_generation=gmax)
        rays, _ = oracle.trace(med, prm, pos, d)
        assert rays["gen"].max() <= gmax
        if gmax == 0:
            assert len(rays) == 1
    # refracted ray into the bottom layer: straight line with Snell angle
    sec = rays[(rays["parent"] == 0) & (rays["seq"] == 0)][0]
    st = 1.5 * math.sin(th) / 1.3
    s_hit = 50.0 / math.cos(th)
    x_hit = s_hit * math.sin(th)
    L = 400.0 - s_hit
    assert np.allclose(sec["pos"], [x_hit + L * st, 0.0, 200.0 + L * math.sqrt(1 - st * st)],
                       atol=1e-8)


def test_earliest_of_two_surfaces_in_one_step(oracle_lib):
    """One step (h = 10 m) that crosses both the surface z = 0 and a stop plane x = 4 m: the
    ray meets the surface first (at x = 2 m), reflects there, and only then reaches the stop
    plane, below the surface.  Straight rays in constant ice, so the geometry is exact."""
    med = {"kind": "layered", "layers": [dict(n0=1.0, absorb=True), dict(z_top=0.0, n0=1.5)]}
    d = np.array([1.0, 0.0, -1.0]) / math.sqrt(2.0)  # 45 degrees upward
    pos = np.array([[0.0], [0.0], [2.0]])
    prm = dict(W.TRACE_DEFAULTS, h0=10.0, max_path=100.0, max_generation=0,
               stop=((1.0, 0.0, 0.0), 4.0))
    rays, _ = oracle.trace(med, prm, pos, d.reshape(3, 1))
    r = rays[0]
    assert r["status"] == oracle.STATUS["REACHED_STOP"] and r["n_refl"] == 1
    assert np.allclose(r["pos"], [4.0, 0.0, 2.0], atol=1e-9)
    assert abs(r["path"] - 4.0 * math.sqrt(2.0)) < 1e-9


def test_receiver_entry_point(oracle_lib):
    med = {"kind": "layered", "layers": [dict(n0=1.7)]}
    pos = np.array([[0.0, 0.0], [0.0, 0.0], [0.0, 0.0]])
    d = np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0]])
    ctr = np.array([[50.0, 0.3, 0.0], [30.0, 0.0, 0.0], [0.0, 70.0, 0.9]])
    rad = np.array([1.0, 2.0, 1.0])
    prm = dict(W.TRACE_DEFAULTS, max_path=100.0)
    rays, hits = oracle.trace(med, prm, pos, d, receivers=(ctr, rad))
    got = sorted((int(h["ray"]), int(h["receiver"]), float(h["path"])) for h in hits)
    want = sorted([(0, 0, 50.0 - math.sqrt(1 - 0.09)), (0, 1, 28.0),
                   (1, 2, 70.0 - math.sqrt(1 - 0.81))])
    assert len(got) == 3
    for g, w in zip(got, want):
        assert g[:2] == w[:2] and abs(g[2] - w[2]) < 1e-9
    for h in hits:
        assert abs(h["time"] - 1.7 * h["path"] / C0) < 1e-18


def test_receiver_hit_carries_the_current_amplitude(oracle_lib):
    """A receiver met before and after a reflection: straight up from 10 m depth in constant
    ice (n 1.5) under absorbing air, a receiver of radius 1 m at 5 m depth.  Entry going up
    at 6 m (path 4 m, amplitude A0), back down after the surface's normal-incidence
    reflection (r = 0.2) at 4 m (path 14 m, amplitude 0.2 A0)."""
    med = {"kind": "layered", "layers": [dict(n0=1.0, absorb=True), dict(z_top=0.0, n0=1.5)]}
    prm = dict(W.TRACE_DEFAULTS, max_path=20.0, max_generation=0)
    rays, hits = oracle.trace(med, prm, np.array([[0.0], [0.0], [10.0]]),
                              np.array([[0.0], [0.0], [-1.0]]), np.array([3.0]),
                              receivers=(np.array([[0.0, 0.0, 5.0]]), np.array([1.0])))
    h = np.sort(hits, order="path")
    assert len(h) == 2
    assert np.allclose(h["path"], [4.0, 14.0], atol=1e-9)
    assert np.allclose(h["amp"], [3.0, 0.6], rtol=1e-12, atol=0)
    assert np.allclose(h["pos"][:, 2], [6.0, 4.0], atol=1e-9)
    assert np.allclose(h["time"], 1.5 * h["path"] / C0, rtol=1e-12, atol=0)


def test_break_conditions(oracle_lib):
    med = {"kind": "layered", "layers": [dict(n0=1.0, absorb=True), dict(z_top=0.0, n0=1.5)]}
    pos = np.array([[0.0], [0.0], [10.5]])
    d = np.array([[0.0], [0.0], [-1.0]])  # straight up: partial reflection at z = 0
    prm = dict(W.TRACE_DEFAULTS, max_path=1e4, max_time=3e-7)
    rays, _ = oracle.trace(med, prm, pos, d)
    assert rays[0]["status"] == oracle.STATUS["MAX_TIME"]
    assert 3e-7 <= rays[0]["time"] < 3e-7 + 10.0 * 1.5 / C0
    prm = dict(W.TRACE_DEFAULTS, max_path=1e4, min_amp=0.5)
    for a0 in (1.0, 4.0, -3.0):
        # the threshold is on A / A0 (Sec. 2, Fig. 1 text): |r| = 0.2 < 0.5 whatever A0 is
        rays, _ = oracle.trace(med, prm, pos, d, np.array([a0]))
        assert rays[0]["status"] == oracle.STATUS["MIN_AMP"], a0
        assert abs(rays[0]["path"] - 10.5) < 1e-9
        assert rays[0]["amp"] == pytest.approx(0.2 * a0, rel=1e-12)
        # the transmitted ray (|t| = 1.2 >= 0.5) is still cast; only weaker ones are not
        sec = rays[rays["parent"] == 0]
        assert len(sec) == 1 and sec[0]["amp"] == pytest.approx(1.2 * a0, rel=1e-12)
    rays, _ = oracle.trace(med, dict(prm, min_amp=1.25), pos, d)
    assert len(rays) == 1  # |t| = 1.2 < 1.25: no secondary


# --------------------------------------------------------------------------------------
# gridded media
# --------------------------------------------------------------------------------------

def test_grid_trilinear_exact_on_linear_field(oracle_lib):
    nx, ny, nz, sp = 6, 5, 7, 2.0
    z, y, x = np.meshgrid(np.arange(nz) * sp, np.arange(ny) * sp, np.arange(nx) * sp,
                          indexing="ij")
    n = (1.3 + 0.01 * x - 0.02 * y + 0.03 * z).astype(np.float32)
    med = oracle.OracleMedium({"kind": "grid", "n": n, "origin": (0.0, 0.0, 0.0), "spacing": sp})
    rng = np.random.default_rng(3)
    for _ in range(50):
        r = rng.uniform(0.0, 8.0, 3)
        val, g = med.eval(r)
        assert abs(val - (1.3 + 0.01 * r[0] - 0.02 * r[1] + 0.03 * r[2])) < 2e-6
        assert np.allclose(g, [0.01, -0.02, 0.03], atol=2e-6)


def test_grid_profile_matches_analytic_tracer(oracle_lib):
    """A grid sampled from the smooth profile reproduces the analytic-medium rays within the
    interpolation error of the sampled profile (h^2/8 max|n''| ~ 1e-4 at 2 m spacing)."""
    sp = 2.0
    ny, nz = 8, 401
    z = np.arange(nz) * sp
    prof = (1.788 - 0.463 * np.exp(-z / 75.0)).astype(np.float32)
    pos, d, a = W.fan_xz(7, 300.0, 30.0, 150.0)
    # a long box in x so that every ray of the fan stays inside it
    nx = 1001
    n = np.empty((nz, ny, nx), np.float32)
    n[:] = prof[:, None, None]
    gmed = {"kind": "grid", "n": n, "origin": (-1000.0, -7.0, 0.0), "spacing": sp}
    prm = dict(W.TRACE_DEFAULTS, tol=1e-7, max_path=300.0, max_generation=0)
    rg, _ = oracle.trace(gmed, prm, pos, d, a)
    ra, _ = oracle.trace(W.single_profile(), prm, pos, d, a)
    assert np.all(rg["status"] == oracle.STATUS["MAX_PATH"])
    assert np.max(np.linalg.norm(rg["pos"] - ra["pos"], axis=1)) < 0.05
    assert np.max(np.abs(rg["time"] - ra["time"])) < 1e-10


def test_grid_leaves_domain(oracle_lib):
    n = np.full((10, 10, 10), 1.5, np.float32)
    gmed = {"kind": "grid", "n": n, "origin": (0.0, 0.0, 0.0), "spacing": 1.0}
    pos = np.array([[4.5], [4.5], [4.5]])
    d = np.array([[1.0], [0.0], [0.0]])
    prm = dict(W.TRACE_DEFAULTS, h_max=1.0, h0=1.0, max_path=100.0)
    rays, _ = oracle.trace(gmed, prm, pos, d)
    assert rays[0]["status"] == oracle.STATUS["LEFT_DOMAIN"]
    assert 9.0 < rays[0]["pos"][0] <= 10.0 + 1e-9


def _optical_length(om, P, sub=40):
    """(1/c0) times the integral of n along the polyline P, Simpson's rule on each segment."""
    T = 0.0
    for a, b in zip(P[:-1], P[1:]):
        u = np.linspace(0.0, 1.0, sub + 1)
        q = a[None, :] + u[:, None] * (b - a)[None, :]
        n = np.array([om.eval(x)[0] for x in q])
        T += np.linalg.norm(b - a) * (n[0] + n[-1] + 4 * n[1:-1:2].sum() + 2 * n[2:-1:2].sum()) \
            / (3 * sub) / C0
    return T


def test_grid_ray_in_random_field_obeys_fermat(oracle_lib):
    """Random-perturbation grid (no closed form): the traced ray is a path of stationary,
    minimal travel time (Fermat).  Points on the ray come from tracing to 40 path lengths; the
    optical length of polylines through them is evaluated with the grid's own (separately
    pinned) interpolation of n.  The ray's first variation under a smooth transverse bump is
    under 2 % of the straight chord's between the same end points (about 0.3 % when right; a
    ray traced through another seed's field, or through the field with its perturbation
    doubled, gives 8-13 %), its second variation is positive, the chord takes longer, and the
    tracer's T equals the ray's optical length."""
    gmed = W.grid_medium(40, 40, 60, spacing=4.0, sigma=5e-3, corr_len=20.0, seed=3)
    om = oracle.OracleMedium(gmed)
    start = np.array([-40.0, -10.0, 40.0])
    th, ph = np.radians(80.0), np.radians(20.0)
    d = np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    S, K = 60.0, 40
    prm = dict(W.TRACE_DEFAULTS, tol=1e-10, h_min=1e-4, h_max=0.5, h0=0.1, max_generation=0)
    pts = [start]
    for k in range(1, K + 1):
        rays, _ = oracle.trace(gmed, dict(prm, max_path=S * k / K), start.reshape(3, 1),
                               d.reshape(3, 1))
        assert rays[0]["status"] == oracle.STATUS["MAX_PATH"]
        pts.append(rays[0]["pos"])
    T_traced = rays[0]["time"]
    ray = np.array(pts)
    s = np.linspace(0.0, 1.0, K + 1)
    chord = ray[0][None, :] + s[:, None] * (ray[-1] - ray[0])[None, :]
    bump = np.sin(np.pi * s)[:, None]
    v = (ray[-1] - ray[0]) / np.linalg.norm(ray[-1] - ray[0])
    u1 = np.cross(v, [0.0, 0.0, 1.0])
    u1 /= np.linalg.norm(u1)
    u2 = np.cross(v, u1)
    E = 0.05
    first, second, T0 = {}, {}, {}
    for name, P in (("ray", ray), ("chord", chord)):
        T0[name] = _optical_length(om, P)
        f, q = [], []
        for u in (u1, u2):
            Tp = _optical_length(om, P + E * bump * u[None, :])
            Tm = _optical_length(om, P - E * bump * u[None, :])
            f.append(abs(Tp - Tm) / 2)
            q.append(Tp + Tm - 2 * T0[name])
        first[name], second[name] = max(f), min(q)
    assert first["ray"] <= 0.02 * first["chord"], (first, second)
    assert second["ray"] > 0.0
    assert T0["ray"] < T0["chord"]
    assert abs(T_traced - T0["ray"]) <= 1e-5 * T_traced


# --------------------------------------------------------------------------------------
# source-receiver path finding: the paper's accuracy study
# --------------------------------------------------------------------------------------

def test_path_finding_reproduces_paper_accuracy(oracle_lib):
    gold = json.load(open(os.path.join(GOLDEN, "paper_accuracy.json")))
    P, acc = gold["profile"], gold["accuracy"]
    prof = ExpProfile(P["n0"], P["dn"], P["z0_m"])
    med = {"kind": "layered", "layers": [
        dict(n0=P["n_above_surface"], absorb=True),
        dict(z_top=0.0, n0=P["n0"], dn=P["dn"], z0=P["z0_m"])]}
    z_s = gold["fig1"]["source_depth_m"]
    L = acc["linear_distance_m"]
    zr = np.array([300.0, 600.0, 900.0, 1200.0])  # receivers outside the shadow zone
    D = np.sqrt(L * L - (zr - z_s) ** 2)
    prm = dict(W.TRACE_DEFAULTS, tol=1e-8, max_path=1e4, max_generation=0)
    count, sol = oracle.find_paths(med, prm, np.full(len(zr), z_s), zr, D,
                                   np.full(len(zr), 512, np.int32), hit_tol=1e-4)
    n_checked = 0
    for i in range(len(zr)):
        ref = solutions(prof, z_s, zr[i], D[i], n_above=P["n_above_surface"])
        assert count[i] == len(ref), (i, count[i], [r["type"] for r in ref])
        for j, r in enumerate(ref):
            s = sol[i, j]
            assert s["type"] == oracle.SOL_TYPE[r["type"]]
            assert abs(math.degrees(s["launch"] - r["launch"])) < acc["launch_angle_deg"]
            # the arrival angle obeys the same Snell invariant: n(z_r) sin(receive) = p
            assert abs(math.degrees(s["receive"] - r["receive"])) < acc["launch_angle_deg"]
            assert abs(s["path"] - r["path"]) < acc["path_length_m"]
            assert abs(s["time"] - r["time"]) < acc["travel_time_s"]
            assert abs(s["amp"] - r["amp"]) < 1e-6
            n_checked += 1
    assert n_checked >= 6


def test_path_finder_matches_closed_forms_on_workload_pairs(oracle_lib):
    """64 pairs of the path-finding workload (its own medium, scan sizes and surface
    reflection) against the closed-form solutions in the Snell invariant: the same solutions
    (count, type), travel times within 1 ps and launch angles within 1e-6 rad at a 0.1 mm
    receiver tolerance.  Two closed-form roots inside one scan interval cannot be bracketed
    by the scan; such roots are left out of the count."""
    cfg = W.paths(64, seed=4)
    P = cfg["pairs"]
    prof = ExpProfile(W.ICE["n0"], W.ICE["dn"], W.ICE["z0"])
    prm = dict(cfg["params"], tol=1e-8)
    count, sol = oracle.find_paths(cfg["medium"], prm, P["zs"], P["zr"], P["dist"],
                                   P["n_angles"], hit_tol=1e-4, max_iter=80)
    n_sol = 0
    for i in range(len(count)):
        ref = solutions(prof, P["zs"][i], P["zr"][i], P["dist"][i], n_above=W.N_AIR)
        dth = math.pi / (P["n_angles"][i] - 1)
        cells = [int(r["launch"] // dth) for r in ref]
        ref = [r for r, c in zip(ref, cells) if cells.count(c) == 1]
        assert count[i] == len(ref), (i, count[i], len(ref))
        for j, r in enumerate(ref):
            s = sol[i, j]
            assert s["type"] == oracle.SOL_TYPE[r["type"]], (i, j)
            assert abs(s["time"] - r["time"]) < 1e-12, (i, j)
            assert abs(s["launch"] - r["launch"]) < 1e-6, (i, j)
            assert abs(s["receive"] - r["receive"]) < 1e-6, (i, j)
            n_sol += 1
    assert n_sol >= 60


def test_path_finder_vertical_pairs(oracle_lib):
    """Receiver straight above or below the source (horizontal distance under the receiver
    tolerance): the one solution is the vertical direct ray, launched down (0) toward a deeper
    receiver and up (pi) toward a shallower one, with T = (1/c0) * integral of n dz =
    (a dz - b zeta (exp(-z1/zeta) - exp(-z2/zeta))) / c0 and path dz."""
    prof = ExpProfile(W.ICE["n0"], W.ICE["dn"], W.ICE["z0"])
    a, b, zeta = prof.a, prof.b, prof.zeta
    med = W.ice_with_surface()
    zs, zr = np.array([100.0, 500.0, 30.0]), np.array([500.0, 100.0, 31.0])
    prm = dict(W.TRACE_DEFAULTS, tol=1e-9, max_generation=0, max_path=1e4)
    count, sol = oracle.find_paths(med, prm, zs, zr, np.zeros(3), np.full(3, 64, np.int32),
                                   hit_tol=1e-4)
    for i in range(3):
        z1, z2 = min(zs[i], zr[i]), max(zs[i], zr[i])
        T = (a * (z2 - z1) - b * zeta * (math.exp(-z1 / zeta) - math.exp(-z2 / zeta))) / C0
        assert count[i] == 1, i
        s = sol[i, 0]
        assert s["type"] == oracle.SOL_TYPE["DIRECT"]
        assert s["launch"] == (0.0 if zr[i] > zs[i] else math.pi)
        assert abs(s["path"] - (z2 - z1)) < 1e-8 and abs(s["time"] - T) < 1e-15, i


def _sphere_medium(n_out, n_in, ctr, R, absorb=False):
    return {"kind": "layered", "layers": [dict(n0=n_out)],
            "spheres": [dict(center=ctr, radius=R, n0=n_in, absorb=absorb)]}


def test_sphere_entry_reflection_refraction_exact(oracle_lib):
    """Straight rays (constant indices) meeting a sphere of higher index: the entry point, the
    reflected primary, the refracted secondary and both amplitudes are exact geometry with the
    local normal (curved boundaries, the paragraph after Fig. 1)."""
    n_out, n_in, R = 1.3, 1.8, 50.0
    ctr = np.array([0.0, 0.0, 500.0])
    med = _sphere_medium(n_out, n_in, ctr, R)
    b = np.array([0.0, 10.0, -25.0, 40.0, 49.0])  # impact parameters in the x-z plane
    n = len(b)
    pos = np.zeros((3, n))
    pos[0] = -200.0
    pos[2] = ctr[2] + b
    d = np.tile(np.array([[1.0], [0.0], [0.0]]), (1, n))
    S = 200.0  # every ray reaches the sphere; no refracted ray reaches the far side
    # a step budget far above the few dozen steps these straight rays need, so that a ray
    # caught at the surface ends (and fails) instead of running on
    prm = dict(W.TRACE_DEFAULTS, tol=1e-9, max_path=S, max_generation=1, max_steps=10_000)
    rays, _ = oracle.trace(med, prm, pos, d)
    for i in range(n):
        xe = -math.sqrt(R * R - b[i] ** 2)
        entry = np.array([xe, 0.0, ctr[2] + b[i]])
        s1 = xe + 200.0
        N = (entry - ctr) / R  # outward normal; the ray comes from outside
        t = np.array([1.0, 0.0, 0.0])
        ci = -t @ N
        t_r = t + 2 * ci * N
        st = (n_out / n_in) ** 2 * (1 - ci * ci)
        ct = math.sqrt(1 - st)
        eta = n_out / n_in
        t_t = eta * t + (eta * ci - ct) * N
        rs = (n_out * ci - n_in * ct) / (n_out * ci + n_in * ct)
        ts = 2 * n_out * ci / (n_out * ci + n_in * ct)
        prim = rays[i]
        assert prim["n_refl"] == 1 and prim["layer"] == 0
        assert np.allclose(prim["pos"], entry + (S - s1) * t_r, atol=1e-7), i
        # landing within eps_b (1e-9 m) of the surface moves the local normal by ~1e-11 rad
        assert abs(prim["amp"] - rs) < 1e-9
        assert abs(prim["time"] - (n_out * S) / C0) < 1e-15
        sec = rays[rays["parent"] == i]
        assert len(sec) == 1
        s = sec[0]
        assert s["gen"] == 1 and s["layer"] == oracle.MAX_LAYERS  # inside sphere 0
        assert abs(s["amp"] - ts) < 1e-9
        assert np.allclose(s["pos"], entry + (S - s1) * t_t, atol=1e-7), i
        assert abs(s["time"] - (n_out * s1 + n_in * (S - s1)) / C0) < 1e-15
        assert np.linalg.norm(s["pos"] - ctr) < R


def test_sphere_exit_into_the_layer_below_and_start_region(oracle_lib):
    """Rays leaving a sphere (n 1.8, radius 50 m, centre at 500 m depth) that sits in the lower
    of two constant layers (n 1.3 above 100 m, 1.5 below) at normal incidence: the
    transmitted ray continues with the index of the layer that holds it (1.5), with
    amplitude 2 n_in / (n_in + n_out).  One starts at the centre, one 1.5 m inside the
    surface: a start point inside the sphere belongs to it however close to the surface."""
    n_in, n_lo = 1.8, 1.5
    ctr = np.array([0.0, 0.0, 500.0])
    med = {"kind": "layered", "layers": [dict(n0=1.3), dict(z_top=100.0, n0=n_lo)],
           "spheres": [dict(center=ctr, radius=50.0, n0=n_in)]}
    S = 90.0  # the reflected primaries do not reach the sphere's far side
    prm = dict(W.TRACE_DEFAULTS, max_path=S, max_generation=1, max_steps=10_000)
    for r0 in (0.0, 48.5):
        pos = (ctr + np.array([r0, 0.0, 0.0])).reshape(3, 1)
        rays, _ = oracle.trace(med, prm, pos, np.array([[1.0], [0.0], [0.0]]))
        sec = rays[rays["parent"] == 0]
        assert len(sec) == 1 and sec[0]["layer"] == 1, r0
        s_exit = 50.0 - r0
        assert abs(sec[0]["amp"] - 2 * n_in / (n_in + n_lo)) < 1e-12
        assert abs(rays[0]["amp"] - (n_in - n_lo) / (n_in + n_lo)) < 1e-12
        assert abs(sec[0]["time"] - (n_in * s_exit + n_lo * (S - s_exit)) / C0) < 1e-15
        assert np.allclose(sec[0]["pos"], ctr + np.array([50.0 + S - s_exit, 0.0, 0.0]),
                           atol=1e-8)


def test_sphere_total_internal_reflection_and_exit(oracle_lib):
    """A ray inside a sphere of higher index: beyond the critical angle it reflects totally
    (amplitude kept, nothing transmitted); at normal incidence it leaves through the surface
    into an absorbing outside only as a transmitted record."""
    n_out, n_in, R = 1.3, 1.8, 50.0
    ctr = np.array([0.0, 0.0, 500.0])
    med = _sphere_medium(n_out, n_in, ctr, R)
    a = 0.8 * R  # sin(incidence) = 0.8 > n_out / n_in = 0.722
    pos = np.array([[0.0], [0.0], [ctr[2] + a]])
    d = np.array([[1.0], [0.0], [0.0]])
    x_hit = math.sqrt(R * R - a * a)
    prm = dict(W.TRACE_DEFAULTS, tol=1e-9, max_path=x_hit + 40.0, max_generation=3,
               max_steps=10_000)
    rays, _ = oracle.trace(med, prm, pos, d)
    assert len(rays) == 1
    r = rays[0]
    hit = np.array([x_hit, 0.0, ctr[2] + a])
    N = (hit - ctr) / R
    t_r = d[:, 0] - 2 * (d[:, 0] @ N) * N
    assert r["n_refl"] == 1 and abs(r["amp"] - 1.0) < 1e-15
    assert np.allclose(r["pos"], hit + 40.0 * t_r, atol=1e-7)
    assert r["layer"] == oracle.MAX_LAYERS
    # from the centre outward: normal incidence into the layer outside
    med2 = {"kind": "layered", "layers": [dict(n0=n_out, absorb=True)],
            "spheres": [dict(center=ctr, radius=R, n0=n_in)]}
    rays, _ = oracle.trace(med2, dict(prm, max_path=120.0), ctr.reshape(3, 1), d)
    sec = rays[rays["parent"] == 0]
    assert len(sec) == 1 and sec[0]["status"] == oracle.STATUS["TRANSMITTED"]
    assert np.allclose(sec[0]["pos"], ctr + R * d[:, 0], atol=1e-8)
    assert abs(sec[0]["amp"] - 2 * n_in / (n_in + n_out)) < 1e-12
    assert abs(rays[0]["amp"] - (n_in - n_out) / (n_in + n_out)) < 1e-12
