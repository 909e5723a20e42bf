"""The GELU of the surrogate's kernels: erf from Abramowitz and Stegun 7.1.26 (Hastings' rational
approximation, absolute error <= 1.5e-7), restated here in numpy (the CUDA code lives in the
library's tensor-core helpers and shares nothing with this file).  Pins: the approximation's
published error bound against math.erf, and GELU and its derivative against their exact forms,
in float64 and in float32 arithmetic (the kernels' precision)."""
import math

import numpy as np

P = 0.3275911
A = (0.254829592, -0.284496736, 1.421413741, -1.453152027, 1.061405429)


def _phi_e(z, dt):
    z = np.asarray(z, dt)
    x = np.abs(z) * dt(0.70710678118654752)
    t = dt(1) / (dt(1) + dt(P) * x)
    p = dt(A[4])
    for a in A[3::-1]:
        p = p * t + dt(a)
    p = p * t
    e = np.exp(-(z * z) * dt(0.5)).astype(dt)
    q = dt(0.5) * p * e
    return np.where(z >= 0, dt(1) - q, q).astype(dt), e


def test_erf_within_the_published_bound():
    x = np.linspace(0.0, 12.0, 200_001)
    phi, _ = _phi_e(x * math.sqrt(2.0), np.float64)
    erf = np.array([math.erf(v) for v in x])
    assert np.max(np.abs((2.0 * phi - 1.0) - erf)) <= 1.5e-7


def test_gelu_and_derivative_in_float32():
    z = np.linspace(-12.0, 12.0, 100_001)
    Phi = 0.5 * (1.0 + np.array([math.erf(v / math.sqrt(2.0)) for v in z]))
    gelu_exact = z * Phi
    dgelu_exact = Phi + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    phi, e = _phi_e(z.astype(np.float32), np.float32)
    zf = z.astype(np.float32)
    gelu = (zf * phi).astype(np.float64)
    dgelu = (phi + zf * e * np.float32(0.39894228040143268)).astype(np.float64)
    # 1.5e-7 / 2 from the approximation of Phi, a few float32 roundings on top
    assert np.max(np.abs(gelu - gelu_exact) / np.maximum(1.0, np.abs(z))) <= 4e-7
    assert np.max(np.abs(dgelu - dgelu_exact)) <= 6e-7
    # far below the BF16 rounding (2^-9 relative) every activation gets before it is used
    assert np.max(np.abs(gelu - gelu_exact) / np.maximum(np.abs(gelu_exact), 1e-3)) < 2.0 ** -12
