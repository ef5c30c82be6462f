"""Pins of the oracle's Algorithms 1-4: invariants, brute-force recounts on
small inputs, the random stream's use, and end-to-end re-validation."""
import numpy as np
import pytest
from scipy import stats

from oracle import kpo
from oracle.kpo import Oracle
from paper_2409_06807_gb300 import workloads as W

VALID, CONTENDER, BERN, WINNER, ACCEPTED, GOAL = 1, 2, 4, 8, 16, 32


def _run_checked(w, n_iters):
    """Iterate with records and check every invariant against the records
    and the exported state (brute force)."""
    o = Oracle(w)
    assert o.reset() == kpo.RUNNING
    prev = o.export()
    for _ in range(n_iters):
        status, st, rec = o.iterate(records=True)
        if status == kpo.FULL:
            break
        cur = o.export()
        n_old, n_new = prev["n_nodes"], cur["n_nodes"]
        ve = np.flatnonzero(prev["in_ve"])
        lam = st["lambda"]
        S = st["n_samples"]
        # Eq. 6 and the sample count
        assert st["n_ve"] == len(ve)
        assert lam == kpo.lam(w.t_e, n_old, len(ve), w.lambda_max)
        assert S == lam * len(ve)
        # sample key -> expanded node
        if S:
            assert np.array_equal(rec["node"], np.repeat(ve, lam))
        fl = rec["flags"]
        valid = (fl & VALID) > 0
        # counters: cumulative and equal to a recount from the records
        dv = cur["n_valid"].astype(np.int64) - prev["n_valid"]
        di = cur["n_invalid"].astype(np.int64) - prev["n_invalid"]
        assert np.array_equal(dv, np.bincount(rec["region"][valid], minlength=len(dv)))
        assert np.array_equal(di, np.bincount(rec["region"][~valid], minlength=len(di)))
        assert dv.sum() + di.sum() == S
        assert np.all(rec["fail_step"][valid] == 0)
        assert np.all((rec["fail_step"][~valid] >= 1) & (rec["fail_step"][~valid] <= rec["k"][~valid]))
        assert np.all((rec["k"] >= w.k_min) & (rec["k"] <= w.k_max))
        # contenders reached a sub-region unvisited at the start of the pass
        cont = (fl & CONTENDER) > 0
        assert np.array_equal(cont, valid & (prev["visited"][rec["sub"]] == 0))
        # one representative (the smallest key) per newly reached sub-region
        win = (fl & WINNER) > 0
        new_subs = np.unique(rec["sub"][cont])
        assert win.sum() == len(new_subs)
        for s in new_subs:
            keys = np.flatnonzero(cont & (rec["sub"] == s))
            assert win[keys[0]] and not win[keys[1:]].any()
        # accepted = valid and (representative or Bernoulli pass)
        acc = (fl & ACCEPTED) > 0
        assert np.array_equal(acc, valid & (win | ((fl & BERN) > 0)))
        # Bernoulli against the previous thresholds, drawn from purpose 1
        for key in np.flatnonzero(valid)[:200]:
            wd = kpo.philox4x32_10([st["iteration"], rec["node"][key], key % lam, 1],
                                   [w.seed & 0xFFFFFFFF, w.seed >> 32])
            assert bool(fl[key] & BERN) == (int(wd[1]) < int(prev["thr"][rec["region"][key]]))
            assert rec["k"][key] == w.k_min + ((int(wd[0]) * (w.k_max - w.k_min + 1)) >> 32)
        # append: ascending key order, parents, regions, visited, |T| <= t_e
        akeys = np.flatnonzero(acc)
        assert n_new == n_old + len(akeys) <= w.t_e
        assert np.array_equal(cur["parent"][n_old:], rec["node"][akeys])
        assert np.array_equal(cur["region"][n_old:], rec["region"][akeys])
        assert np.array_equal(cur["sub"][n_old:], rec["sub"][akeys])
        np.testing.assert_array_equal(cur["state"][n_old:], rec["state"][akeys])
        assert np.all(cur["parent"][1:] < np.arange(1, n_new))
        vis = prev["visited"].copy()
        vis[rec["sub"][akeys]] = 1
        assert np.array_equal(cur["visited"], vis)
        # Cov = visited sub-regions per region; R_avail = regions with a node
        per = w.n_sub_per
        assert np.array_equal(cur["cov"], cur["visited"].reshape(-1, per).sum(1))
        av = np.zeros_like(cur["avail"])
        av[cur["region"][:n_new]] = 1
        assert np.array_equal(cur["avail"], av)
        # every newly reached sub-region gained exactly one node
        assert np.all(np.bincount(cur["sub"][n_old:], minlength=len(vis))[new_subs] >= 1)
        # estimates: P >= eps on R_avail (Lemma 1), P = 1 elsewhere
        _, p, _ = o.estimates()
        assert np.all(p[cur["avail"] == 1] >= w.eps)
        assert np.all(p[cur["avail"] == 0] == 1.0)
        # node sets: old nodes by one draw each (purpose 2), new nodes in V_E
        assert np.all(cur["in_ve"][n_old:] == 1)
        for v in range(min(n_old, 300)):
            wd = kpo.philox4x32_10([st["iteration"], v, 0, 2], [w.seed & 0xFFFFFFFF, w.seed >> 32])
            assert cur["in_ve"][v] == (int(wd[0]) < int(cur["thr"][cur["region"][v]]))
        # goal: smallest new node id inside the ball
        goal = (fl & GOAL) > 0
        assert np.all(goal <= acc)
        if goal.any():
            assert st["goal_node"] == n_old + np.flatnonzero(akeys == np.flatnonzero(goal)[0])[0]
            assert status == kpo.SOLVED
        prev = cur
        if status != kpo.RUNNING:
            break
    return o


@pytest.mark.parametrize("system", [W.DI, W.DUBINS, W.QUAD])
def test_invariants_tiny(system):
    for seed in range(3):
        _run_checked(W.tiny(system, seed=seed), 12)


def test_invariants_c1_small_frontier():
    _run_checked(W.c1(1, t_e=6000), 6)


def test_tree_full_stops():
    """Eq. 6 gives lambda = 0 once t_e - |T| < |V_E|: the loop stops."""
    o = Oracle(W.tiny(W.DI, seed=1, t_e=40, goal_r=np.float32(0.0)))
    o.reset()
    status, _ = o.run(100)
    assert status == kpo.FULL and o.n_nodes <= 40


def test_root_in_goal_and_invalid_root():
    w = W.tiny(W.DI)
    o = Oracle(w.with_(goal_c=w.x_init[:3].copy()))
    assert o.reset() == kpo.SOLVED and list(o.path()) == [0]
    bad = w.x_init.copy()
    bad[3] = 5.0  # velocity outside its bound
    assert Oracle(w).reset(bad) == kpo.ERR


def test_determinism_and_seed_dependence():
    a, b, c = Oracle(W.c1(0)), Oracle(W.c1(0)), Oracle(W.c1(0).with_(seed=1))
    for o in (a, b, c):
        o.reset()
        o.run(4)
    ea, eb, ec = a.export(), b.export(), c.export()
    assert ea["n_nodes"] == eb["n_nodes"] and np.array_equal(ea["state"], eb["state"])
    assert ea["n_nodes"] != ec["n_nodes"] or not np.array_equal(ea["state"], ec["state"])


def test_node_selection_rate_matches_p_accept():
    """Each old node enters V_E with probability P_accept of its region."""
    o = Oracle(W.c1(2))
    o.reset()
    o.run(4)
    before = o.export()
    o.iterate()
    after = o.export()
    n_old = before["n_nodes"]
    p = after["thr"][before["region"][:n_old]].astype(np.float64) / 2 ** 32
    sel = after["in_ve"][:n_old].astype(np.float64)
    z = (sel.sum() - p.sum()) / np.sqrt((p * (1 - p)).sum())
    assert abs(z) < 5
    # finer: nodes grouped by P decile
    order = np.argsort(p)
    for chunk in np.array_split(order, 5):
        e, v = p[chunk].sum(), (p[chunk] * (1 - p[chunk])).sum()
        assert abs(sel[chunk].sum() - e) < 5 * np.sqrt(v) + 1


def test_control_and_duration_draws_are_uniform():
    w = W.c1(0)
    o = Oracle(w)
    o.reset()
    o.run(2)
    _, st, rec = o.iterate(records=True)
    u = W.np.asarray(rec["uraw"], np.uint64)
    assert stats.kstest((u[:, :3] >> 8).ravel() / 2 ** 24, "uniform").pvalue > 1e-4
    counts = np.bincount(rec["k"], minlength=w.k_max + 1)[w.k_min:]
    assert stats.chisquare(counts).pvalue > 1e-4


@pytest.mark.parametrize("make,seed", [(W.c1, 0), (W.c1, 4)])
def test_solution_revalidated(make, seed):
    """A returned trajectory: re-propagating every edge from its parent's
    stored state reproduces the child, the edge passes the dense check, and
    the last state lies in the goal ball (Problem 1)."""
    w = make(seed)
    o = Oracle(w)
    o.reset()
    status, _ = o.run(60)
    assert status == kpo.SOLVED
    t = o.export()
    path = o.path()
    assert path[0] == 0 and t["parent"][path[1]] == 0
    for a, b in zip(path, path[1:]):
        assert t["parent"][b] == a
        depth, x_end = o.dense_check(t["state"][a], t["ctrl"][b], t["steps"][b], 100)
        assert depth <= 0.0
        np.testing.assert_allclose(x_end, t["state"][b], atol=1e-12)
    g = t["state"][path[-1], :3]
    assert np.linalg.norm(g - w.goal_c) <= w.goal_r
