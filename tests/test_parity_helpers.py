"""The helpers the GPU parity tests rely on (tests/parity.py), on the CPU: rays are matched by
their place in the split tree whatever order the secondaries come in, identical records pass,
and a moved end point, a missing subtree or swapped siblings fail."""
import numpy as np
import pytest

import oracle
from paper_1810_01780_gb300 import workloads as W
from parity import (check_fp64, check_within, match, oracle_rays, sensitive_keys,
                    subset_by_roots, subtree_of_roots, tilt, tree_keys)


@pytest.fixture(scope="module")
def rays(oracle_lib):
    cfg = W.batched(n=300, seed=11)
    ref, _ = oracle.trace(cfg["medium"], cfg["params"], *cfg["rays"])
    o = oracle_rays(ref)
    assert (o["generation"] >= 2).any()  # secondaries of secondaries
    return o, cfg["params"]["tol"], 300


def _shuffled(o, n_prim, seed):
    """The same records with the secondaries in another order that keeps every parent before
    its secondaries (by generation, random within one), parents renumbered."""
    rng = np.random.default_rng(seed)
    sec = np.arange(n_prim, len(o["parent"]))
    order = np.concatenate([np.arange(n_prim),
                            sec[np.lexsort((rng.random(len(sec)), o["generation"][sec]))]])
    new_of = np.empty_like(order)
    new_of[order] = np.arange(len(order))
    g = {k: v[order].copy() for k, v in o.items()}
    g["parent"] = np.where(g["parent"] < 0, -1, new_of[np.maximum(g["parent"], 0)])
    return g


def test_identical_records_in_another_order_match(rays):
    o, tol, n = rays
    g = _shuffled(o, n, 1)
    assert not np.array_equal(g["pos"], o["pos"])  # really reordered
    gi, oi, only_g, only_o = match(g, o)
    assert not only_g and not only_o and len(gi) == len(o["path"])
    for k in o:
        if k != "parent":
            np.testing.assert_array_equal(g[k][gi], o[k][oi], err_msg=k)
    assert check_fp64(g, o, tol) == 1.0


def test_a_moved_end_point_fails(rays):
    o, tol, n = rays
    g = _shuffled(o, n, 2)
    j = len(g["path"]) - 1
    g["pos"][j] += 1e-6 * (g["path"][j] + 1.0) * np.array([1.0, 0.0, 0.0]) * 5
    with pytest.raises(AssertionError):
        check_fp64(g, o, tol)


def test_a_missing_subtree_fails(rays):
    o, tol, n = rays
    g = _shuffled(o, n, 3)
    last = len(g["path"]) - 1  # a ray of the last generation: no secondaries of its own
    keep = np.arange(len(g["path"])) != last
    h = {k: v[keep] for k, v in g.items()}
    gi, oi, only_g, only_o = match(h, o)
    assert not only_g and len(only_o) == 1
    with pytest.raises(AssertionError):
        check_fp64(h, o, tol)


def test_swapped_siblings_fail(rays):
    o, tol, n = rays
    g = _shuffled(o, n, 4)
    # two secondaries of one parent, cast at different splits
    par = g["parent"]
    for p in np.unique(par[par >= 0]):
        kids = np.nonzero(par == p)[0]
        if len(kids) >= 2 and g["path"][kids[0]] != g["path"][kids[1]]:
            a, b = kids[:2]
            break
    else:
        pytest.skip("no parent with two secondaries")
    g["seq"][[a, b]] = g["seq"][[b, a]]
    with pytest.raises(AssertionError):
        check_fp64(g, o, tol)


def test_subtrees_and_tilt(rays):
    o, _, n = rays
    idx, root = subtree_of_roots(o["parent"], np.array([3, 7]))
    assert set(root[idx]) == {3, 7} and 3 in idx and 7 in idx
    others = np.setdiff1d(np.arange(len(root)), idx)
    assert not np.isin(root[others], [3, 7]).any()
    d = W.isotropic_dirs(np.random.default_rng(0), 1000)
    t = tilt(d, 1e-3, 5)
    assert np.allclose(np.linalg.norm(t, axis=0), 1.0, atol=1e-12)
    assert np.allclose(np.arccos(np.clip((t * d).sum(0), -1, 1)), 1e-3, rtol=1e-5)


def test_subset_by_roots_rekeys_like_an_oracle_run_on_the_roots(rays, oracle_lib):
    """The subtrees of sampled roots, cut from a run over all primaries (in shuffled order),
    match an oracle run on those primaries alone, record for record."""
    o, tol, n = rays
    g = _shuffled(o, n, 5)
    roots = np.array([2, 5, 11, 40, 299])
    sub, take = subset_by_roots(g, roots)
    cfg = W.batched(n=300, seed=11)
    ref, _ = oracle.trace(cfg["medium"], cfg["params"], *W.subsample(cfg["rays"], roots))
    r = oracle_rays(ref)
    assert len(sub["path"]) == len(r["path"])
    gi, oi, only_g, only_o = match(sub, r)
    assert not only_g and not only_o
    for k in ("pos", "time", "status", "generation", "n_acc"):
        np.testing.assert_array_equal(sub[k][gi], r[k][oi], err_msg=k)


def test_check_within_excuses_only_ill_conditioned_rays(rays):
    """check_within: identical records pass; a ray moved beyond the tolerance fails unless it
    or an ancestor is in the ill-conditioned set; a status change and a missing ray likewise."""
    o, tol, n = rays
    g = _shuffled(o, n, 6)
    assert check_within(g, o, set()) == (len(o["path"]), 0)
    keys = tree_keys(g["parent"], g["seq"])
    j = int(np.nonzero(g["generation"] == 2)[0][0])
    parent_key = keys[j][:-1]
    moved = {k: v.copy() for k, v in g.items()}
    moved["pos"][j] += np.array([0.0, 2e-3, 0.0])
    with pytest.raises(AssertionError):
        check_within(moved, o, set())
    assert check_within(moved, o, {parent_key})[1] >= 1  # excused through its parent
    late = {k: v.copy() for k, v in g.items()}
    late["time"][j] += 2e-11
    with pytest.raises(AssertionError):
        check_within(late, o, set())
    flipped = {k: v.copy() for k, v in g.items()}
    flipped["status"][j] = 3 if flipped["status"][j] != 3 else 1
    with pytest.raises(AssertionError):
        check_within(flipped, o, set())
    check_within(flipped, o, {keys[j]})
    keep = np.arange(len(g["path"])) != len(g["path"]) - 1  # drop a last-generation ray
    gone = {k: v[keep] for k, v in g.items()}
    lost = keys[len(g["path"]) - 1]
    with pytest.raises(AssertionError):
        check_within(gone, o, set())
    check_within(gone, o, {lost})


def test_sensitive_keys_flags_rays_that_move_under_a_tilt(rays):
    o, tol, n = rays
    g = _shuffled(o, n, 7)
    assert sensitive_keys(o, g) == set()
    keys = tree_keys(g["parent"], g["seq"])
    h = {k: v.copy() for k, v in g.items()}
    h["pos"][4] += 5e-3
    h["status"][9] = 9
    assert sensitive_keys(o, h) == {keys[4], keys[9]}


def test_step_capped_keys_checks_the_excuse(rays):
    """A ray capped (status 7) in one run only is excused when the other run got at least as
    far along it (accepted steps and reflections); one that stopped short fails; rays capped in
    both runs are excused as they are."""
    from parity import step_capped_keys

    o, _, _ = rays
    ko = tree_keys(o["parent"], o["seq"])
    g = {k: v.copy() for k, v in o.items()}
    assert step_capped_keys(g, o) == set()
    o2 = {k: v.copy() for k, v in o.items()}
    o2["status"][0] = 7  # capped in the reference only, the other run equally far: excused
    o2["status"][1] = 7
    g["status"][1] = 7  # capped in both
    assert step_capped_keys(g, o2) == {ko[0], ko[1]}
    g["n_acc"][0] = o2["n_acc"][0] - 1  # the uncapped run stopped short of the capped one
    with pytest.raises(AssertionError):
        step_capped_keys(g, o2)
