"""The closed forms of the exponential profile against adaptive quadrature and geometry.

These closed forms pin the oracle; here they are pinned themselves, independently of any
ray-tracing code: by Gauss-Kronrod quadrature of the defining integrals (Snell invariant
p = n sin(theta) in a stratified medium) and by limiting cases."""
import math

import numpy as np
import pytest

from oracle.analytic import C0, ExpProfile, solutions


@pytest.mark.parametrize("p", [0.05, 0.6, 1.1, 1.3, 1.6])
def test_branch_closed_form_vs_quadrature(p):
    prof = ExpProfile()
    for z1, z2 in [(200.0, 1500.0), (50.0, 900.0), (1000.0, 300.0)]:
        if p >= float(prof.n(min(z1, z2))):
            continue
        cf = prof.branch(z1, z2, p)
        q = prof.quad_branch(z1, z2, p)
        for a, b in zip(cf, q):
            assert abs(a - b) <= 1e-10 * abs(b) + 1e-20


def test_turning_branch_vs_quadrature():
    prof = ExpProfile()
    p = 1.5
    zt = prof.turning_depth(p)
    assert abs(float(prof.n(zt)) - p) < 1e-14
    cf = prof.branch(zt, 400.0, p)
    q = prof.quad_branch(zt, 400.0, p)
    for a, b in zip(cf, q):
        assert abs(a - b) <= 1e-9 * abs(b)


def test_uniform_limit_is_straight_line():
    # b -> 0: straight ray, X = dz tan(theta), S = dz / cos(theta), T = n S / c0
    prof = ExpProfile(a=1.5, b=1e-9, zeta=75.0)
    th = math.radians(35.0)
    p = 1.5 * math.sin(th)
    X, S, T = prof.branch(100.0, 600.0, p)
    assert abs(X - 500.0 * math.tan(th)) < 1e-5
    assert abs(S - 500.0 / math.cos(th)) < 1e-5
    assert abs(T - 1.5 * S / C0) < 1e-13


def test_solution_families_hit_the_receiver():
    prof = ExpProfile(1.788, 0.463, 71.4)
    for zs, zr, D in [(240.0, 900.0, 1300.0), (240.0, 600.0, 1400.0), (800.0, 100.0, 900.0)]:
        sols = solutions(prof, zs, zr, D)
        assert sols, (zs, zr, D)
        for s in sols:
            th = s["launch"]
            assert abs(float(prof.n(zs)) * math.sin(th) - s["p"]) < 1e-12
            assert s["path"] > math.hypot(D, zr - zs) - 1e-9  # never shorter than the chord
        times = [s["time"] for s in sols]
        assert times == sorted(times)
