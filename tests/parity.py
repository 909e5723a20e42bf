"""Helpers for comparing CUDA-path outputs with the oracle (test infrastructure).

Secondary rays are created in a non-deterministic order on the GPU, so rays are matched by
their position in the split tree: a primary is keyed by its index, a secondary by its
parent's key plus the index of the split on the parent that cast it."""
from __future__ import annotations

import numpy as np


def gpu_rays(res) -> dict:
    r = res["rays"]
    out = {
        "pos": r["end_pos"].cpu().numpy().T.copy(),
        "dir": r["end_dir"].cpu().numpy().T.copy(),
    }
    for k in ("path", "time", "amp", "status", "generation", "seq", "layer", "parent", "n_acc",
              "n_rej", "n_root", "n_refl", "n_turn"):
        out[k] = r[k].cpu().numpy()
    return out


def oracle_rays(rays) -> dict:
    return {
        "pos": rays["pos"], "dir": rays["dir"], "path": rays["path"], "time": rays["time"],
        "amp": rays["amp"], "status": rays["status"], "generation": rays["gen"],
        "seq": rays["seq"], "layer": rays["layer"], "parent": rays["parent"],
        "n_acc": rays["n_acc"], "n_rej": rays["n_rej"], "n_root": rays["n_root"],
        "n_refl": rays["n_refl"], "n_turn": rays["n_turn"],
    }


def tree_keys(parent, seq):
    """Key of every ray; a parent always has a smaller index than its secondaries."""
    keys = []
    for i in range(len(parent)):
        p = int(parent[i])
        if p < 0:
            keys.append((i,))
        else:
            assert p < i, (i, p)
            keys.append(keys[p] + (int(seq[i]),))
    return keys


def match(g: dict, o: dict):
    """Index arrays (gi, oi) of rays present in both, plus the unmatched key sets."""
    kg = tree_keys(g["parent"], g["seq"])
    ko = tree_keys(o["parent"], o["seq"])
    mo = {k: i for i, k in enumerate(ko)}
    gi, oi, only_g = [], [], []
    for i, k in enumerate(kg):
        j = mo.pop(k, None)
        if j is None:
            only_g.append(k)
        else:
            gi.append(i)
            oi.append(j)
    return np.array(gi, dtype=np.int64), np.array(oi, dtype=np.int64), only_g, list(mo.keys())


def errors(g, o, gi, oi):
    dp = np.linalg.norm(g["pos"][gi] - o["pos"][oi], axis=1)
    dd = np.linalg.norm(g["dir"][gi] - o["dir"][oi], axis=1)
    ds = np.abs(g["path"][gi] - o["path"][oi])
    dT = np.abs(g["time"][gi] - o["time"][oi])
    dA = np.abs(g["amp"][gi] - o["amp"][oi])
    return dp, dd, ds, dT, dA


def same_steps(g, o, gi, oi):
    return (g["n_acc"][gi] == o["n_acc"][oi]) & (g["n_rej"][gi] == o["n_rej"][oi])


def subtree_of_roots(parent, roots):
    """Indices of every ray whose root primary is in `roots` (primaries are 0..n-1)."""
    n = len(parent)
    root = np.empty(n, dtype=np.int64)
    for i in range(n):
        j = i
        while parent[j] >= 0:
            j = int(parent[j])
        root[i] = j
    return np.nonzero(np.isin(root, roots))[0], root


def check_fp64(g, o, tol, min_tier1=0.95, rel=1e-9):
    gi, oi, only_g, only_o = match(g, o)
    assert not only_g and not only_o, (len(only_g), len(only_o))
    assert np.array_equal(g["status"][gi], o["status"][oi])
    assert np.array_equal(g["generation"][gi], o["generation"][oi])
    dp, dd, ds, dT, dA = errors(g, o, gi, oi)
    s = o["path"][oi]
    same = same_steps(g, o, gi, oi)
    t1 = same
    assert np.all(dp[t1] <= rel * (s[t1] + 1.0)), dp[t1].max()
    assert np.all(ds[t1] <= rel * (s[t1] + 1.0)), ds[t1].max()
    assert np.all(dT[t1] <= rel * o["time"][oi][t1] + 1e-18), dT[t1].max()
    assert np.all(dd[t1] <= rel), dd[t1].max()
    assert np.all(dA[t1] <= rel), dA[t1].max()
    assert same.mean() >= min_tier1, same.mean()
    t2 = ~same
    if t2.any():
        assert np.all(dp[t2] <= 10 * tol * (s[t2] + 1.0)), dp[t2].max()
        assert np.all(dT[t2] <= 10 * tol * o["time"][oi][t2] + 1e-15)
    return same.mean()


def tilt(d, angle, seed):
    """Rotate every direction by `angle` rad about a random axis perpendicular to it."""
    from paper_1810_01780_gb300.workloads import tilted_dirs

    return tilted_dirs(d, angle, seed)


def subset_by_roots(g: dict, roots) -> tuple[dict, np.ndarray]:
    """The rays of a GPU run that descend from the primaries `roots` (sorted indices), re-keyed
    so that they compare with an oracle run on those primaries alone: primaries first, in root
    order, then the secondaries in their order of creation, parents renumbered.  Returns the
    subset and the GPU indices it was taken from (in the subset's order)."""
    roots = np.asarray(roots)
    gsel, groot = subtree_of_roots(g["parent"], roots)
    rank = {int(r): i for i, r in enumerate(roots)}
    order = np.argsort([rank[int(groot[j])] if g["parent"][j] < 0 else 10**12 + j for j in gsel],
                       kind="stable")
    take = gsel[order]
    new_of = {int(old): new for new, old in enumerate(take)}
    sub = {k: v[take] for k, v in g.items()}
    sub["parent"] = np.array([-1 if p < 0 else new_of[int(p)] for p in sub["parent"]],
                             dtype=np.int64)
    return sub, take


def sensitive_keys(o: dict, o_tilted: dict, pos_tol=1e-3, time_tol=1e-11) -> set:
    """Split-tree keys of the rays whose result moves by more than (pos_tol, time_tol), or
    changes status, or disappears, when every launch direction is tilted by a tiny angle:
    there the problem itself is ill-conditioned (grazing or critical incidence, an amplitude
    at its threshold), and two correct computations may differ by more than the tolerance."""
    oi, ti, only_o, _ = match(o, o_tilted)
    ko = tree_keys(o["parent"], o["seq"])
    dp = np.linalg.norm(o["pos"][oi] - o_tilted["pos"][ti], axis=1)
    dT = np.abs(o["time"][oi] - o_tilted["time"][ti])
    moved = (o["status"][oi] != o_tilted["status"][ti]) | (dp > pos_tol) | (dT > time_tol)
    return {ko[i] for i in oi[moved]} | set(only_o)


def step_capped_keys(g: dict, o: dict) -> set:
    """Split-tree keys of the rays that ran into the attempted-step cap (status 7) in either
    run.  Rejected steps and the root-finding iterations of boundary landings count against
    the cap, and their number differs between two precisions, so where the cap falls on a ray
    that needs about that many attempts is arbitrary: such a ray is excused like an
    ill-conditioned one.  The excuse is checked: where only one run was capped, the other got
    at least as far along the same ray (at least as many accepted steps and reflections)."""
    gi, oi, _, _ = match(g, o)
    ko = tree_keys(o["parent"], o["seq"])
    cg, co = g["status"][gi] == 7, o["status"][oi] == 7
    ahead_g = (g["n_acc"][gi] >= o["n_acc"][oi]) & (g["n_refl"][gi] >= o["n_refl"][oi])
    ahead_o = (o["n_acc"][oi] >= g["n_acc"][gi]) & (o["n_refl"][oi] >= g["n_refl"][gi])
    bad = (cg & ~co & ~ahead_o) | (co & ~cg & ~ahead_g)
    assert not bad.any(), [(ko[i], int(g["n_acc"][j]), int(o["n_acc"][i]))
                           for j, i in zip(gi[bad], oi[bad])][:5]
    return {ko[i] for i in oi[cg | co]}


def excused(key, sens: set) -> bool:
    """True if the ray `key` or one of its ancestors is ill-conditioned (in `sens`)."""
    return any(key[:m] in sens for m in range(1, len(key) + 1))


def check_within(g: dict, o: dict, sens: set, pos_tol=1e-3, time_tol=1e-11):
    """Element-by-element check of a run `g` against a reference `o`: every ray of `o` that is
    not excused by `sens` exists in `g` with the same status and generation, its end point
    within pos_tol and its travel time within time_tol; a ray of `g` absent from `o` must be
    excused.  Returns (number of rays checked, number excused)."""
    gi, oi, only_g, only_o = match(g, o)
    bad_g = [k for k in only_g if not excused(k, sens)]
    bad_o = [k for k in only_o if not excused(k, sens)]
    assert not bad_g and not bad_o, (bad_g[:5], bad_o[:5])
    ko = tree_keys(o["parent"], o["seq"])
    wc = np.array([not excused(ko[i], sens) for i in oi], dtype=bool)
    gi, oi = gi[wc], oi[wc]
    st = g["status"][gi] == o["status"][oi]
    assert st.all(), [(ko[i], g["status"][j], o["status"][i]) for j, i in zip(gi[~st], oi[~st])][:5]
    assert np.array_equal(g["generation"][gi], o["generation"][oi])
    dp, dd, ds, dT, dA = errors(g, o, gi, oi)
    far = (dp > pos_tol) | (dT > time_tol)
    assert not far.any(), [(ko[i], float(p), float(t)) for i, p, t in
                           zip(oi[far], dp[far], dT[far])][:5]
    return len(gi), int((~wc).sum()) + len(only_o)
