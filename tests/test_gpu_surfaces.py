"""Non-horizontal boundaries on the GPU (boundary shapes beyond the plane, Sec. 2, the paragraph
after Fig. 1): a tilted ice surface carrying a height field of undulations and a tilted
internal boundary, through the C ABI (rp_trace) against the FP64 oracle.

Tolerances: FP64 as for the planes (1e-9 relative for rays whose step sequence equals the
oracle's, 10 tol s for the others, same statuses and split trees); FP32-mixed against FP64: every
ray within 1 mm and 0.01 ns with the same status, unless the FP64 result of the ray or of an
ancestor moves by more than that under a 1e-7 rad launch tilt (at most 1 % of the rays)."""
import math

import numpy as np
import pytest

import oracle
from oracle.analytic import C0
from parity import check_fp64, check_within, gpu_rays, oracle_rays, sensitive_keys, tilt
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


def test_surfaces_fp64_matches_oracle(rp):
    cfg = W.surfaces()
    rays = W.subsample(cfg["rays"], np.arange(3000))
    med = rp.Medium(cfg["medium"])
    g = gpu_rays(rp.trace(med, *rays, params=cfg["params"], precision="fp64"))
    ref, _ = oracle.trace(cfg["medium"], cfg["params"], *rays)
    o = oracle_rays(ref)
    assert (o["n_refl"] > 0).sum() > 500 and (o["generation"] >= 2).any()
    frac = check_fp64(g, o, cfg["params"]["tol"])
    print("surfaces fp64 vs oracle: %d rays, tier-1 fraction %.4f" % (len(o["path"]), frac))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tilted_plane_exact_geometry_on_the_gpu(rp, precision):
    """The oracle pin's exact geometry (constant layers n = 1.5 below, 1.0 above a tilted plane):
    reflected end point, refracted end point, amplitudes, travel time."""
    N = np.array([0.25, -0.15, 1.0])
    N /= np.linalg.norm(N)
    n1, n2, z0, S = 1.5, 1.0, 100.0, 400.0
    med = {"kind": "layered", "layers": [dict(n0=n2), dict(z_top=z0, n0=n1)],
           "surfaces": [dict(layer=1, normal=tuple(N))]}
    t = np.array([0.3, 0.1, -1.0])
    t /= np.linalg.norm(t)
    p0 = np.array([10.0, 20.0, 180.0])
    res = gpu_rays(rp.trace(rp.Medium(med), p0[:, None], t[:, None],
                            params=dict(W.TRACE_DEFAULTS, max_path=S), precision=precision))
    lam = N @ (np.array([0.0, 0.0, z0]) - p0) / (N @ t)
    hit = p0 + lam * t
    ci = -(t @ N)
    t_r = t - 2 * (t @ N) * N
    ct = math.sqrt(1 - (n1 / n2) ** 2 * (1 - ci * ci))
    t_t = (n1 / n2) * t + ((n1 / n2) * ci - ct) * N
    rs = (n1 * ci - n2 * ct) / (n1 * ci + n2 * ct)
    ts = 2 * n1 * ci / (n1 * ci + n2 * ct)
    tol = 1e-7 if precision == "fp64" else 2e-4
    assert len(res["path"]) == 2 and res["parent"][1] == 0
    assert np.allclose(res["pos"][0], hit + (S - lam) * t_r, atol=tol)
    assert np.allclose(res["pos"][1], hit + (S - lam) * t_t, atol=tol)
    assert abs(res["amp"][0] - rs) < 1e-6 and abs(res["amp"][1] - ts) < 1e-6
    assert abs(res["time"][0] - n1 * S / C0) < (1e-17 if precision == "fp64" else 1e-12)
    assert abs(res["time"][1] - (n1 * lam + n2 * (S - lam)) / C0) < \
        (1e-17 if precision == "fp64" else 1e-12)


def test_surfaces_fp32_mixed_vs_fp64(rp):
    cfg = W.surfaces()
    pos, d, a = W.subsample(cfg["rays"], np.arange(20000))
    med = rp.Medium(cfg["medium"])
    g64 = gpu_rays(rp.trace(med, pos, d, a, params=cfg["params"], precision="fp64"))
    g32 = gpu_rays(rp.trace(med, pos, d, a, params=cfg["params"], precision="fp32"))
    gt = gpu_rays(rp.trace(med, pos, tilt(d, 1e-7, 9), a, params=cfg["params"],
                           precision="fp64"))
    sens = sensitive_keys(g64, gt)
    n_checked, n_excused = check_within(g32, g64, sens)
    n = len(g64["path"])
    print("surfaces fp32 vs fp64: %d checked, %d ill-conditioned (%.4f), %d excused (%.4f)" % (
        n_checked, len(sens), len(sens) / n, n_excused, n_excused / n))
    assert len(sens) <= 0.01 * n and n_excused <= 0.025 * n


def test_surface_media_validation(rp):
    from paper_1810_01780_gb300._abi import RPError

    base = W.two_layer_ice()
    bad = [dict(layer=0, normal=(0, 0, 1)), dict(layer=3, normal=(0, 0, 1)),
           dict(layer=1, normal=(0.1, 0, -1)),
           dict(layer=1, normal=(0, 0, 1), height=np.zeros((1, 4)), origin=(0, 0),
                spacing=(1, 1)),
           dict(layer=1, normal=(0, 0, 1), height=np.zeros((3, 3)), origin=(0, 0),
                spacing=(0, 1)),
           dict(layer=1, normal=(0, 0, 1), height=np.full((3, 3), np.nan), origin=(0, 0),
                spacing=(1, 1))]
    for srf in bad:
        with pytest.raises(RPError) as e:
            rp.Medium(dict(base, surfaces=[srf]))
        assert e.value.code == -1, srf
    with pytest.raises(RPError) as e:  # one boundary, two surfaces
        rp.Medium(dict(base, surfaces=[dict(layer=1, normal=(0, 0, 1))] * 2))
    assert e.value.code == -1
    with pytest.raises(RPError) as e:  # spheres and surfaces together
        rp.Medium(dict(W.ice_with_inclusions(), surfaces=[dict(layer=1, normal=(0, 0, 1))]))
    assert e.value.code == -5
    # path finding takes horizontal boundaries only
    med = rp.Medium(W.rough_ice())
    with pytest.raises(RPError):
        rp.find_paths(med, [100.0], [50.0], [300.0], np.array([32], np.int32),
                      W.paths()["params"], "fp64")
