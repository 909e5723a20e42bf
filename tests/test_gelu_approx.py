"""The GELU of the surrogate's kernels: the normal distribution function Phi from Abramowitz and
Stegun 26.2.17 (Hastings' rational approximation, absolute error < 7.5e-8), restated here in
numpy (the CUDA code lives in the library's tensor-core helpers and shares nothing with this
file).  Pins: the approximation's published error bound against math.erf, and GELU and its
derivative against their exact forms, in float64 and in float32 arithmetic (the kernels'
precision)."""
import math

import numpy as np

P = 0.2316419
B = (0.319381530, -0.356563782, 1.781477937, -1.821255978, 1.330274429)


def _phi_d(z, dt):
    """(Phi(z), phi(z)) in arithmetic of type dt: 1 - Phi(|z|) = phi(z) t (b1 + ... + b5 t^4)."""
    z = np.asarray(z, dt)
    t = dt(1) / (dt(1) + dt(P) * np.abs(z))
    p = dt(B[4])
    for b in B[3::-1]:
        p = p * t + dt(b)
    p = p * t
    # the density as one power of two, as the kernels take it
    d = np.exp2((z * z) * dt(-0.72134752044448170) + dt(-1.3257480647361594)).astype(dt)
    q = p * d
    return np.where(z >= 0, dt(1) - q, q).astype(dt), d


def _phi_exact(x):
    return np.array([0.5 * (1.0 + math.erf(v / math.sqrt(2.0))) for v in x])


def test_phi_within_the_published_bound():
    x = np.linspace(-12.0, 12.0, 240_001)
    phi, d = _phi_d(x, np.float64)
    assert np.max(np.abs(phi - _phi_exact(x))) < 7.5e-8
    # the density itself is exact up to rounding
    assert np.max(np.abs(d - np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi))) < 1e-15


def test_symmetry_and_special_values():
    x = np.linspace(1e-3, 9.0, 9_000)  # x > 0: -x takes the other branch
    a, _ = _phi_d(x, np.float64)
    b, _ = _phi_d(-x, np.float64)
    assert np.max(np.abs(a + b - 1.0)) < 1e-15  # Phi(x) + Phi(-x) = 1 by construction
    half, _ = _phi_d(np.array([0.0]), np.float64)
    assert abs(half[0] - 0.5) < 7.5e-8


def test_gelu_and_derivative_in_float32():
    z = np.linspace(-12.0, 12.0, 100_001)
    Phi = _phi_exact(z)
    gelu_exact = z * Phi
    dgelu_exact = Phi + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    zf = z.astype(np.float32)
    phi, d = _phi_d(zf, np.float32)
    gelu = (zf * phi).astype(np.float64)
    dgelu = (phi + zf * d).astype(np.float64)
    # 7.5e-8 from the approximation of Phi, a few float32 roundings on top
    assert np.max(np.abs(gelu - gelu_exact) / np.maximum(1.0, np.abs(z))) <= 4e-7
    assert np.max(np.abs(dgelu - dgelu_exact)) <= 6e-7
    # far below the BF16 rounding (2^-9 relative) every activation gets before it is used
    assert np.max(np.abs(gelu - gelu_exact) / np.maximum(np.abs(gelu_exact), 1e-3)) < 2.0 ** -12
