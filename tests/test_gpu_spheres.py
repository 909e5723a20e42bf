"""Curved boundaries (the paragraph after Fig. 1): spherical inclusions in the layered ice on the
GPU.  FP64 path against the oracle with the tolerances of test_gpu_trace; FP32-mixed against
FP64 within 1 mm / 0.01 ns for every ray whose FP64 result is stable under a 1e-7 rad launch
tilt; exact geometry at a constant-index sphere on both paths; validation of the medium."""
import math

import numpy as np
import pytest

import oracle
from parity import (check_fp64, check_within, errors, gpu_rays, match,
                    oracle_rays, sensitive_keys, step_capped_keys, tilt)
from paper_1810_01780_gb300 import workloads as W

pytestmark = pytest.mark.gpu
C0 = 299792458.0


@pytest.fixture(scope="module")
def rp():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1810_01780_gb300 import build

    build.build()
    import paper_1810_01780_gb300 as rp

    return rp


def _run(rp, medium, params, rays, precision):
    pos, d, a = rays
    return gpu_rays(rp.trace(rp.Medium(medium), pos, d, a, params=params, precision=precision))


def test_spheres_fp64_matches_oracle(rp):
    cfg = W.spheres(4096)
    g = _run(rp, cfg["medium"], cfg["params"], cfg["rays"], "fp64")
    ref, _ = oracle.trace(cfg["medium"], cfg["params"], *cfg["rays"])
    o = oracle_rays(ref)
    assert len(g["path"]) == len(ref)
    frac = check_fp64(g, o, cfg["params"]["tol"])
    print("tier-1 fraction", frac)
    inside = g["layer"] >= oracle.MAX_LAYERS
    assert inside.sum() > 100  # rays end inside both inclusions
    assert set(np.unique(g["layer"][inside])) == {oracle.MAX_LAYERS, oracle.MAX_LAYERS + 1}


def test_spheres_fp32_mixed_vs_fp64(rp):
    """FP32-mixed against FP64, ray by ray: every ray that is not excused as ill-conditioned
    (its FP64 result, or an ancestor's, moves by more than 1 mm / 0.01 ns, changes status or
    disappears when every launch direction is tilted by 1e-7 rad, in either of two independent
    tilt directions) exists in both runs with the
    same status and generation, within 1 mm and 0.01 ns.  At most 5 % of the rays are
    ill-conditioned or excused with their secondaries.  Rays that reach the workload's cap of
    1,000 attempted steps in either run are excused too: rays trapped in the lens by total
    internal reflection spend the budget on the root iterations of about a hundred landings,
    whose number differs between the precisions; where only one run was capped the other must
    have got at least as far along the ray.  At most 0.2 % of the rays."""
    cfg = W.spheres(65536)
    pos, d, a = cfg["rays"]
    g64 = _run(rp, cfg["medium"], cfg["params"], (pos, d, a), "fp64")
    g32 = _run(rp, cfg["medium"], cfg["params"], (pos, d, a), "fp32")
    # behind reflections off a convex sphere the sensitivity depends on the tilt's direction:
    # a ray is ill-conditioned if either of two independent 1e-7 rad tilts moves it
    sens = set()
    for seed in (5, 11):
        gpt = _run(rp, cfg["medium"], cfg["params"], (pos, tilt(d, 1e-7, seed), a), "fp64")
        sens |= sensitive_keys(g64, gpt)
    capped = step_capped_keys(g32, g64)
    n_checked, n_excused = check_within(g32, g64, sens | capped)
    n = len(g64["path"])
    assert len(capped) <= 0.002 * n
    gi, oi, _, _ = match(g32, g64)
    dp, dd, ds, dT, dA = errors(g32, g64, gi, oi)
    print("spheres fp32 vs fp64: %d rays checked, %d ill-conditioned (%.4f), %d excused with their "
          "secondaries (%.4f); p50/p99 |dr| %.2e/%.2e m" % (
              n_checked, len(sens), len(sens) / n, n_excused, n_excused / n, np.median(dp),
              np.quantile(dp, 0.99)))
    assert len(sens) <= 0.05 * n and n_excused <= 0.05 * n
    assert n_checked >= 0.9 * n


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_constant_sphere_exact_geometry(rp, precision):
    """Straight rays meeting a sphere of higher constant index: reflected primary and refracted
    secondary against the exact geometry with the local normal (as the oracle's pin)."""
    n_out, n_in, R = 1.3, 1.8, 50.0
    ctr = np.array([0.0, 0.0, 500.0])
    med = {"kind": "layered", "layers": [dict(n0=n_out)],
           "spheres": [dict(center=ctr, radius=R, n0=n_in)]}
    b = np.array([0.0, 10.0, -25.0, 40.0, 49.0])
    n = len(b)
    pos = np.zeros((3, n))
    pos[0] = -200.0
    pos[2] = ctr[2] + b
    d = np.tile(np.array([[1.0], [0.0], [0.0]]), (1, n))
    S = 200.0
    # the FP32-mixed error estimate has a rounding floor near 1e-7 per step: a tolerance
    # below it would force every step down to h_min
    prm = dict(W.TRACE_DEFAULTS, tol=1e-9 if precision == "fp64" else 1e-6, max_path=S,
               max_generation=1)
    g = _run(rp, med, prm, (pos, d, np.ones(n)), precision)
    assert np.all(g["status"] == 1)  # MAX_PATH
    tol_x = 1e-7 if precision == "fp64" else 2e-5
    tol_t = 1e-14 if precision == "fp64" else 1e-12
    for i in range(n):
        xe = -math.sqrt(R * R - b[i] ** 2)
        entry = np.array([xe, 0.0, ctr[2] + b[i]])
        s1 = xe + 200.0
        N = (entry - ctr) / R
        t = np.array([1.0, 0.0, 0.0])
        ci = -t @ N
        ct = math.sqrt(1 - (n_out / n_in) ** 2 * (1 - ci * ci))
        eta = n_out / n_in
        t_r = t + 2 * ci * N
        t_t = eta * t + (eta * ci - ct) * N
        rs = (n_out * ci - n_in * ct) / (n_out * ci + n_in * ct)
        ts = 2 * n_out * ci / (n_out * ci + n_in * ct)
        assert g["n_refl"][i] == 1
        assert np.allclose(g["pos"][i], entry + (S - s1) * t_r, atol=tol_x), i
        assert abs(g["amp"][i] - rs) < 1e-6
        sec = np.nonzero(g["parent"] == i)[0]
        assert len(sec) == 1
        j = sec[0]
        assert g["layer"][j] == oracle.MAX_LAYERS and g["generation"][j] == 1
        assert abs(g["amp"][j] - ts) < 1e-6
        assert np.allclose(g["pos"][j], entry + (S - s1) * t_t, atol=tol_x), i
        assert abs(g["time"][j] - (n_out * s1 + n_in * (S - s1)) / C0) < tol_t


def test_sphere_media_validation(rp):
    from paper_1810_01780_gb300._abi import RPError

    base = W.ice_with_surface()
    cut = dict(base, spheres=[dict(center=(0, 0, 10.0), radius=20.0, n0=1.5)])  # crosses z = 0
    with pytest.raises(RPError):
        rp.Medium(cut)
    overlap = dict(base, spheres=[dict(center=(0, 0, 300.0), radius=30.0, n0=1.5),
                                  dict(center=(40, 0, 300.0), radius=20.0, n0=1.5)])
    with pytest.raises(RPError):
        rp.Medium(overlap)
    med = rp.Medium(W.ice_with_inclusions())
    with pytest.raises(RPError):  # the path finder covers layered media without spheres
        rp.find_paths(med, [500.0], [100.0], [300.0], [64], W.paths(1)["params"], "fp32")
