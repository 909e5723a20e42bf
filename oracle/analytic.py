"""Closed-form ray solutions of the exponential ice profile (test infrastructure).

The profile n(z) = a - b exp(-z/zeta) of Sec. 2 (Fig. 1 text, accuracy study) is
stratified, so along every ray the Snell invariant p = n(z) sin(theta) is constant
(theta measured from the +z axis, z = depth).  With u = exp(-z/zeta) and
w(u) = sqrt((a - b u)^2 - p^2) the horizontal range, arc length and travel time of a branch
on which z is monotonic are

    X  = zeta p | I1(u1) - I1(u2) |
    S  = zeta | a dI1 - b dI0 |
    cT = zeta | a^2 dI1 - 2 a b dI0 + b^2 dIu |

with the elementary antiderivatives (tables of integrals of R = A u^2 + B u + C,
A = b^2, B = -2ab, C = a^2 - p^2 > 0):

    I1(u) = int du / (u w) = -(1/c) ln((2 c^2 - 2 a b u + 2 c w) / u),     c = sqrt(C)
    I0(u) = int du / w     = -(1/b) ln(n + w),                             n = a - b u
    Iu(u) = int u du / w   = w / b^2 + (a / b) I0(u)

A ray launched upward turns where w = 0, i.e. n(z_t) = p.  ``quad_branch`` evaluates the same
three integrals by adaptive quadrature in z so that the closed forms are not trusted blindly.

Parity: pinned by adaptive Gauss-Kronrod quadrature of the same integrals (with the
turning-point substitution), the b -> 0 straight-line limit, and solutions that, traced by
the oracle, hit their receivers (tests/test_analytic_pins.py).

This module is test infrastructure: only tests, the smoke check and the benchmark's CPU
baseline import it.
"""
from __future__ import annotations

import math

import numpy as np

C0 = 299792458.0


class ExpProfile:
    """n(z) = a - b exp(-z / zeta), z = depth (positive downward)."""

    def __init__(self, a=1.788, b=0.463, zeta=75.0):
        self.a, self.b, self.zeta = float(a), float(b), float(zeta)

    def n(self, z):
        return self.a - self.b * np.exp(-np.asarray(z, dtype=np.float64) / self.zeta)

    # ---- antiderivatives in u -------------------------------------------------------
    def _w(self, u, p):
        if u is None:  # the turning point itself: w = 0 exactly
            return 0.0
        n = self.a - self.b * u
        return math.sqrt(max(n * n - p * p, 0.0))

    def _u(self, z, p):
        """u = exp(-z/zeta); None marks the turning depth (n(z) = p), where w vanishes."""
        return None if z == self.turning_depth(p) else math.exp(-z / self.zeta)

    def _uv(self, u, p):
        return (self.a - p) / self.b if u is None else u

    def _I1(self, u, p):
        a, b = self.a, self.b
        c = math.sqrt(a * a - p * p)
        w, u = self._w(u, p), self._uv(u, p)
        return -(1.0 / c) * math.log(abs(2.0 * c * c - 2.0 * a * b * u + 2.0 * c * w) / u)

    def _I0(self, u, p):
        w, u = self._w(u, p), self._uv(u, p)
        n = p if w == 0.0 else self.a - self.b * u
        return -(1.0 / self.b) * math.log(n + w)

    def _Iu(self, u, p):
        return self._w(u, p) / (self.b * self.b) + (self.a / self.b) * self._I0(u, p)

    def branch(self, z1, z2, p):
        """(X, S, T) along a monotonic branch between depths z1 and z2."""
        a, b, zeta = self.a, self.b, self.zeta
        u1, u2 = self._u(z1, p), self._u(z2, p)
        d1 = self._I1(u1, p) - self._I1(u2, p)
        d0 = self._I0(u1, p) - self._I0(u2, p)
        du = self._Iu(u1, p) - self._Iu(u2, p)
        X = zeta * p * abs(d1)
        S = zeta * abs(a * d1 - b * d0)
        T = zeta * abs(a * a * d1 - 2.0 * a * b * d0 + b * b * du) / C0
        return X, S, T

    def turning_depth(self, p):
        """Depth where n(z) = p (the ray turns); +inf if p >= a."""
        if p >= self.a:
            return math.inf
        return -self.zeta * math.log((self.a - p) / self.b)

    def quad_branch(self, z1, z2, p):
        """Same as ``branch`` by adaptive Gauss-Kronrod quadrature in z (independent check).

        The inverse-square-root singularity at a turning point is removed with the
        substitution z = z_t + sign * v^2."""
        from scipy.integrate import quad

        zt = self.turning_depth(p)
        lo, hi = min(z1, z2), max(z1, z2)

        def fx(z):
            n = self.n(z)
            return p / math.sqrt(n * n - p * p)

        def fs(z):
            n = self.n(z)
            return n / math.sqrt(n * n - p * p)

        def ft(z):
            n = self.n(z)
            return n * n / math.sqrt(n * n - p * p) / C0

        touches = math.isfinite(zt) and abs(lo - zt) < 1e-9 * max(1.0, abs(zt))
        out = []
        for f in (fx, fs, ft):
            if touches:
                V = math.sqrt(hi - zt)
                g = lambda v, f=f: f(zt + v * v) * 2.0 * v
                val, _ = quad(g, 0.0, V, epsabs=0.0, epsrel=1e-13, limit=200)
            else:
                val, _ = quad(f, lo, hi, epsabs=0.0, epsrel=1e-13, limit=200)
            out.append(val)
        return tuple(out)

    # ---- a whole ray from a launch -------------------------------------------------------
    def ray_to_depth(self, z_s, theta0, z_end, ends_down=True):
        """(X, S, T) of the ray launched at depth z_s with angle theta0 (from +z) when it is
        at depth z_end; for an upward launch the ray may have turned (ends_down=True) or not.
        The medium is the single profile continued to all z (no surface)."""
        p = float(self.n(z_s)) * math.sin(theta0)
        if math.cos(theta0) >= 0.0:
            return self.branch(z_s, z_end, p)
        if not ends_down:
            return self.branch(z_s, z_end, p)
        zt = self.turning_depth(p)
        x1, s1, t1 = self.branch(z_s, zt, p)
        x2, s2, t2 = self.branch(zt, z_end, p)
        return x1 + x2, s1 + s2, t1 + t2


def fresnel_rs(n1, n2, cos_i):
    """s-polarised amplitude reflection (|r| = 1 beyond the critical angle, phase dropped)."""
    s2 = (n1 / n2) ** 2 * (1.0 - cos_i * cos_i)
    if s2 > 1.0:
        return 1.0
    ct = math.sqrt(1.0 - s2)
    return (n1 * cos_i - n2 * ct) / (n1 * cos_i + n2 * ct)


def solutions(prof: ExpProfile, z_s, z_r, D, n_above=1.0, n_p=4000):
    """All source-receiver solutions in the profile with a reflecting surface at z = 0
    (medium of index n_above above it).  Returns a list of dicts sorted by travel time:
    type, p, launch, receive, time, path, amp.

    Each solution family (direct, refracted through a turning point, surface-reflected)
    gives the range X(p); roots of X(p) = D are bracketed on a fine p grid and polished by
    Brent's method."""
    from scipy.optimize import brentq

    a = prof.a
    n_s, n_r, n_0 = float(prof.n(z_s)), float(prof.n(z_r)), float(prof.n(0.0))
    zmin = min(z_s, z_r)
    out = []

    def add(kind, p, X, S, T, launch_up, recv_up, amp=1.0):
        launch = math.asin(min(1.0, p / n_s))
        launch = math.pi - launch if launch_up else launch
        recv = math.asin(min(1.0, p / n_r))
        recv = math.pi - recv if recv_up else recv
        out.append(dict(type=kind, p=p, launch=launch, receive=recv, time=T, path=S, amp=amp))

    def direct(p):
        return prof.branch(z_s, z_r, p)

    def refracted(p):
        zt = prof.turning_depth(p)
        x1 = prof.branch(z_s, zt, p)
        x2 = prof.branch(zt, z_r, p)
        return tuple(u + v for u, v in zip(x1, x2))

    def reflected(p):
        x1 = prof.branch(z_s, 0.0, p)
        x2 = prof.branch(0.0, z_r, p)
        return tuple(u + v for u, v in zip(x1, x2))

    eps = 1e-12
    fams = [
        ("DIRECT", direct, 0.0, min(n_s, n_r) * (1 - eps)),
        ("REFRACTED", refracted, n_0 * (1 + eps), float(prof.n(zmin)) * (1 - eps)),
        ("REFLECTED", reflected, 0.0, n_0 * (1 - eps)),
    ]
    for kind, fam, plo, phi in fams:
        if not phi > plo:
            continue
        ps = np.linspace(plo, phi, n_p)
        xs = np.array([fam(p)[0] - D for p in ps])
        for i in range(n_p - 1):
            if np.sign(xs[i]) == 0:
                continue
            if np.sign(xs[i]) != np.sign(xs[i + 1]):
                p = brentq(lambda q: fam(q)[0] - D, ps[i], ps[i + 1], xtol=1e-15, rtol=1e-15)
                X, S, T = fam(p)
                if kind == "DIRECT":
                    up = z_r < z_s
                    add(kind, p, X, S, T, up, up)
                elif kind == "REFRACTED":
                    add(kind, p, X, S, T, True, False)
                else:
                    cos_i = math.sqrt(max(0.0, 1.0 - (p / n_0) ** 2))
                    add(kind, p, X, S, T, True, False, fresnel_rs(n_0, n_above, cos_i))
    out.sort(key=lambda d: d["time"])
    return out
