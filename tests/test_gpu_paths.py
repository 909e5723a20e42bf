"""CUDA path finder (rp_find_paths) vs the FP64 oracle and the closed-form solutions.

Tolerances: FP64 path vs oracle -- same solution count per pair; a solution found after the
same number of bisection steps has the same launch angle (both bisect the same FP64 bracket)
to 1e-12 rad, travel time to 1e-9 relative and path length to 1e-5 m.  FP32-mixed vs the
oracle or FP64: the same counts and types, every solution's travel time at the receiver (the
hit moved by its miss along the eikonal gradient) within 0.01 ns, path length within 1 mm when
the bisection took the same steps.  The paper's accuracy claim (Sec. 2: launch angle 0.01 deg, path 0.005 m, time
7 ps at 1500 m) is checked against the closed forms on the GPU as on the oracle."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle.analytic import ExpProfile, solutions
from paper_1810_01780_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def rp():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1810_01780_gb300 import build

    build.build()
    import paper_1810_01780_gb300 as rp

    return rp


def _np(res):
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in res.items()}


def _time_at_receiver(sol, i, j, zr, medium):
    """Travel time of solution j of pair i moved from where the ray crosses the receiver plane
    (z_r + miss) to the receiver itself, with the eikonal's gradient along that plane,
    dT/dz = n(z_r) cos(receive angle) / c0 (ray optics: grad T = n t / c0).  Two valid hits of
    one solution, a few centimetres apart, then agree to second order in their misses."""
    ice = medium["layers"][1]
    n = ice["n0"] - ice["dn"] * math.exp(-max(zr, 0.0) / ice["z0"])
    return sol["time"][i, j] - sol["miss"][i, j] * n * math.cos(sol["receive"][i, j]) / 299792458.0


def _compare_all(g, o, zr, medium, t_abs, hit_tol):
    """Every pair: the same solution count; every solution: the same type, both misses below
    hit_tol, travel times at the receiver within t_abs.  Returns the number of solutions and
    how many of them converged after a different number of bisection steps."""
    assert np.array_equal(g["count"], o["count"]), np.nonzero(g["count"] != o["count"])[0][:10]
    n_sol = n_other = 0
    for i in range(len(o["count"])):
        for j in range(o["count"][i]):
            assert g["type"][i, j] == o["type"][i, j], (i, j)
            assert abs(g["miss"][i, j]) < hit_tol and abs(o["miss"][i, j]) < hit_tol, (i, j)
            dt = abs(_time_at_receiver(g, i, j, zr[i], medium) -
                     _time_at_receiver(o, i, j, zr[i], medium))
            assert dt <= t_abs, (i, j, dt)
            n_sol += 1
            n_other += int(g["n_iter"][i, j] != o["n_iter"][i, j])
    return n_sol, n_other


def _oracle_sol(medium, params, zs, zr, D, na, **kw):
    oc, osol = oracle.find_paths(medium, params, zs, zr, D, na, **kw)
    return {"count": oc, **{k: osol[k] for k in ("type", "n_iter", "launch", "receive", "time",
                                                  "path", "miss")}}


def test_paths_fp64_match_oracle(rp):
    """96 pairs of the workload at their full scan resolution (32..512 angles), FP64: the same
    solutions as the oracle -- counts and types; a solution found after the same number of
    bisection steps (both bisect the same FP64 bracket) with the same launch angle to 1e-12 rad,
    travel time to 1e-9 relative and path length to 1e-5 m; every solution's travel time at the
    receiver within 1 ps."""
    cfg = W.paths()
    P = cfg["pairs"]
    idx = np.arange(96)
    zs, zr, D, na = P["zs"][idx], P["zr"][idx], P["dist"][idx], P["n_angles"][idx]
    assert na.max() > 400 and na.min() < 100
    g = _np(rp.find_paths(rp.Medium(cfg["medium"]), zs, zr, D, na, cfg["params"], "fp64"))
    o = _oracle_sol(cfg["medium"], cfg["params"], zs, zr, D, na)
    assert o["count"].sum() > 50
    n_sol, n_other = _compare_all(g, o, zr, cfg["medium"], 1e-12, cfg["hit_tol"])
    assert n_other == 0
    for i in range(len(idx)):
        for j in range(o["count"][i]):
            assert abs(g["launch"][i, j] - o["launch"][i, j]) <= 1e-12, (i, j)
            assert abs(g["time"][i, j] - o["time"][i, j]) <= 1e-9 * o["time"][i, j], (i, j)
            assert abs(g["path"][i, j] - o["path"][i, j]) <= 1e-5, (i, j)
    print("paths fp64 vs oracle: %d pairs, %d solutions" % (len(idx), n_sol))


def test_paths_fp32_vs_fp64(rp):
    """4,000 pairs of the workload, FP32-mixed against FP64 on the GPU: the same solution counts
    and types, every solution's travel time at the receiver within 10 ps; where the bisection
    took the same steps, the same launch angle (the FP64 bisection of the same bracket) and path
    lengths within 1 mm."""
    cfg = W.paths()
    P = cfg["pairs"]
    idx = np.arange(4000)
    args = (P["zs"][idx], P["zr"][idx], P["dist"][idx], P["n_angles"][idx])
    med = rp.Medium(cfg["medium"])
    g64 = _np(rp.find_paths(med, *args, cfg["params"], "fp64"))
    g32 = _np(rp.find_paths(med, *args, cfg["params"], "fp32"))
    n_sol, n_other = _compare_all(g32, g64, P["zr"][idx], cfg["medium"], 1e-11, cfg["hit_tol"])
    for i in range(len(idx)):
        for j in range(g64["count"][i]):
            if g32["n_iter"][i, j] == g64["n_iter"][i, j]:
                assert g32["launch"][i, j] == g64["launch"][i, j], (i, j)
                assert abs(g32["path"][i, j] - g64["path"][i, j]) <= 1e-3, (i, j)
    print("paths fp32 vs fp64: %d solutions, %d after a different number of bisection steps" % (
        n_sol, n_other))
    assert n_other <= 0.02 * n_sol and n_sol > 1000


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_paths_reproduce_paper_accuracy(rp, precision):
    gold = json.load(open(os.path.join(GOLDEN, "paper_accuracy.json")))
    Pp, acc = gold["profile"], gold["accuracy"]
    prof = ExpProfile(Pp["n0"], Pp["dn"], Pp["z0_m"])
    med = {"kind": "layered", "layers": [
        dict(n0=Pp["n_above_surface"], absorb=True),
        dict(z_top=0.0, n0=Pp["n0"], dn=Pp["dn"], z0=Pp["z0_m"])]}
    z_s = gold["fig1"]["source_depth_m"]
    L = acc["linear_distance_m"]
    zr = np.array([300.0, 600.0, 900.0, 1200.0])
    D = np.sqrt(L * L - (zr - z_s) ** 2)
    prm = dict(W.TRACE_DEFAULTS, tol=1e-8, max_generation=0)
    g = _np(rp.find_paths(rp.Medium(med), np.full(4, z_s), zr, D, np.full(4, 512, np.int32), prm,
                          precision, hit_tol=1e-4))
    n = 0
    for i in range(4):
        ref = solutions(prof, z_s, zr[i], D[i], n_above=Pp["n_above_surface"])
        assert g["count"][i] == len(ref)
        for j, r in enumerate(ref):
            assert abs(math.degrees(g["launch"][i, j] - r["launch"])) < acc["launch_angle_deg"]
            assert abs(g["path"][i, j] - r["path"]) < acc["path_length_m"]
            assert abs(g["time"][i, j] - r["time"]) < acc["travel_time_s"]
            n += 1
    assert n >= 6


def test_paths_full_size_sampled(rp):
    """All 65,536 pairs in one call (FP32-mixed, the benchmark's configuration); 96 sampled pairs
    against the FP64 oracle at their full scan resolution: the same solution counts and types,
    every solution's travel time at the receiver within 10 ps, path lengths within 1 mm where
    the bisection took the same steps."""
    cfg = W.paths()
    P = cfg["pairs"]
    g = _np(rp.find_paths(rp.Medium(cfg["medium"]), P["zs"], P["zr"], P["dist"], P["n_angles"],
                          cfg["params"], "fp32"))
    assert g["stats"]["rays"] > 10_000_000
    rng = np.random.default_rng(7)
    idx = np.sort(rng.choice(len(P["zs"]), 96, replace=False))
    o = _oracle_sol(cfg["medium"], cfg["params"], P["zs"][idx], P["zr"][idx], P["dist"][idx],
                    P["n_angles"][idx])
    sub = {k: v[idx] for k, v in g.items() if k != "stats"}
    n_sol, n_other = _compare_all(sub, o, P["zr"][idx], cfg["medium"], 1e-11, cfg["hit_tol"])
    for i in range(len(idx)):
        for j in range(o["count"][i]):
            if sub["n_iter"][i, j] == o["n_iter"][i, j]:
                assert abs(sub["path"][i, j] - o["path"][i, j]) <= 1e-3, (i, j)
    print("paths full size fp32 vs oracle: %d solutions, %d after a different number of "
          "bisection steps" % (n_sol, n_other))
    assert n_sol > 60


def test_paths_vertical_and_edge_pairs(rp):
    cfg = W.paths()
    zs = np.array([500.0, 100.0, 300.0, 0.0])
    zr = np.array([150.0, 180.0, 300.0, 50.0])
    D = np.array([0.01, 0.0, 2000.0, 10.0])
    na = np.array([64, 64, 2, 128], dtype=np.int32)
    g = _np(rp.find_paths(rp.Medium(cfg["medium"]), zs, zr, D, na, cfg["params"], "fp64"))
    oc, osol = oracle.find_paths(cfg["medium"], cfg["params"], zs, zr, D, na)
    assert np.array_equal(g["count"], oc)
    for i in range(2):  # vertical pairs: straight up / down, T = integral of n dz / c0
        assert g["count"][i] == 1 and g["type"][i, 0] == 0
        assert abs(g["time"][i, 0] - osol[i, 0]["time"]) < 1e-18


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_speculative_bisection_equals_per_lane_bisection(rp, precision):
    """A batch with few brackets per lane takes speculative rounds of several bisection steps
    (one tree of midpoints per bracket per round); a full batch bisects one bracket per lane.
    The pairs of a small batch, solved alone and inside the full batch, give identical
    solutions field by field."""
    cfg = W.paths()
    P = cfg["pairs"]
    kw = dict(hit_tol=0.005, max_iter=cfg["max_iter"], max_sol=cfg["max_sol"])
    med = rp.Medium(cfg["medium"])
    full = _np(rp.find_paths(med, P["zs"], P["zr"], P["dist"], P["n_angles"], cfg["params"],
                             precision, **kw))
    sub = np.arange(0, len(P["zs"]), 97)[:512]
    small = _np(rp.find_paths(med, P["zs"][sub], P["zr"][sub], P["dist"][sub],
                              P["n_angles"][sub], cfg["params"], precision, **kw))
    assert small["stats"]["waves"] > 2 and full["stats"]["waves"] == 2  # rounds vs per lane
    np.testing.assert_array_equal(small["count"], full["count"][sub])
    for k in ("type", "n_iter", "launch", "receive", "time", "path", "amp", "miss"):
        np.testing.assert_array_equal(small[k], full[k][sub], err_msg=k)
