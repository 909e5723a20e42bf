"""CUDA path finder (rp_find_paths) vs the FP64 oracle and the closed-form solutions.

Tolerances: FP64 path vs oracle -- same solution count per pair; a solution found after the
same number of bisection steps has the same launch angle (both bisect the same FP64 bracket)
to 1e-12 rad, travel time and path length to 1e-9 relative.  FP32-mixed vs FP64: launch angle
identical when the bisection took the same steps, travel time within 0.01 ns and path length
within 1 mm.  The paper's accuracy claim (Sec. 2: launch angle 0.01 deg, path 0.005 m, time
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


def _compare(g, ocount, osol, max_sol, ang_tol, t_rel, s_abs, min_match=0.99):
    n = len(ocount)
    same_count = g["count"] == ocount
    assert same_count.mean() >= min_match, same_count.mean()
    checked = 0
    for i in np.nonzero(same_count)[0]:
        for j in range(ocount[i]):
            o = osol[i, j]
            assert g["type"][i, j] == o["type"], (i, j)
            if g["n_iter"][i, j] != o["n_iter"]:
                continue  # converged one bisection step apart: a different valid hit
            assert abs(g["launch"][i, j] - o["launch"]) <= ang_tol, (i, j)
            assert abs(g["time"][i, j] - o["time"]) <= t_rel * o["time"] + 1e-18, (i, j)
            assert abs(g["path"][i, j] - o["path"]) <= s_abs, (i, j)
            checked += 1
    return checked


def test_paths_fp64_match_oracle(rp):
    cfg = W.paths()
    P = cfg["pairs"]
    idx = np.arange(160)
    zs, zr, D, na = P["zs"][idx], P["zr"][idx], P["dist"][idx], P["n_angles"][idx]
    na = np.minimum(na, 96).astype(np.int32)  # keep the oracle run short
    g = _np(rp.find_paths(rp.Medium(cfg["medium"]), zs, zr, D, na, cfg["params"], "fp64"))
    oc, osol = oracle.find_paths(cfg["medium"], cfg["params"], zs, zr, D, na)
    assert oc.sum() > 50
    checked = _compare(g, oc, osol, 4, 1e-12, 1e-9, 1e-9 * 1e4)
    assert checked > 40


def test_paths_fp32_vs_fp64(rp):
    cfg = W.paths()
    P = cfg["pairs"]
    idx = np.arange(4000)
    args = (P["zs"][idx], P["zr"][idx], P["dist"][idx], P["n_angles"][idx])
    med = rp.Medium(cfg["medium"])
    g64 = _np(rp.find_paths(med, *args, cfg["params"], "fp64"))
    g32 = _np(rp.find_paths(med, *args, cfg["params"], "fp32"))
    same = g32["count"] == g64["count"]
    assert same.mean() >= 0.99
    n_same_iter = n_total = 0
    for i in np.nonzero(same)[0]:
        for j in range(g64["count"][i]):
            n_total += 1
            assert g32["type"][i, j] == g64["type"][i, j]
            if g32["n_iter"][i, j] != g64["n_iter"][i, j]:
                continue
            n_same_iter += 1
            assert g32["launch"][i, j] == g64["launch"][i, j]
            assert abs(g32["time"][i, j] - g64["time"][i, j]) <= 1e-11
            assert abs(g32["path"][i, j] - g64["path"][i, j]) <= 1e-3
    assert n_same_iter >= 0.98 * n_total and n_total > 1000


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
    """All 65,536 pairs in one call (FP32-mixed); 48 sampled pairs against the oracle."""
    cfg = W.paths()
    P = cfg["pairs"]
    g = _np(rp.find_paths(rp.Medium(cfg["medium"]), P["zs"], P["zr"], P["dist"], P["n_angles"],
                          cfg["params"], "fp32"))
    assert g["stats"]["rays"] > 10_000_000
    rng = np.random.default_rng(7)
    idx = np.sort(rng.choice(len(P["zs"]), 48, replace=False))
    oc, osol = oracle.find_paths(cfg["medium"], cfg["params"], P["zs"][idx], P["zr"][idx],
                                 P["dist"][idx], P["n_angles"][idx])
    sub = {k: v[idx] for k, v in g.items() if k != "stats"}
    _compare(sub, oc, osol, 4, 1e-6, 1e-6, 1e-3, min_match=0.95)


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
