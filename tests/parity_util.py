"""Element-wise comparison of one loop pass of the CUDA planner with the
oracle on the same inputs.

Tolerances (spec contract):
  * integers (Philox words, k, node ids, regions, sub-regions, flags,
    counters, thresholds, node sets, appended nodes) must match exactly;
  * propagated states within 1e-4 after normalising each dimension by its
    bound range;
  * a sample's validity, region or sub-region may differ only when the
    oracle puts it within TAU = 1e-4 (normalised) of the decision boundary:
    its hull-vs-box or state-bound clearance, its distance to a cell face
    (or to the goal sphere).  The FP32 device path and the FP64 oracle take
    these decisions on states that differ by rounding, so the decision is
    only defined up to that margin.
"""
import numpy as np

TAU = 1e-4
STATE_TOL = 1e-4


def state_scale(w):
    lo = np.asarray(w.x_lo[: w.d], np.float64)
    hi = np.asarray(w.x_hi[: w.d], np.float64)
    s = hi - lo
    return np.where(np.isfinite(s) & (s > 0), s, 1.0)


def compare_pass(w, ost, orec, gst, grec, expect_exact=None, before=None, after=None,
                 otree=None, vol=None):
    """Compare one pass.  Returns the number of samples whose decisions
    differ (all of them ambiguous, else AssertionError).

    With the device's trees around the pass (before, after), the oracle's
    tree after it (otree) and the region volumes of Eq. 3 (vol), everything
    the pass decides downstream of the expand is also checked, whether or
    not an ambiguous sample flipped: see check_downstream."""
    assert gst["n_ve"] == ost["n_ve"], (gst, ost)
    assert gst["lambda"] == ost["lambda"], (gst, ost)
    S = ost["n_samples"]
    assert gst["n_samples"] == S
    if S == 0:
        return 0
    assert np.array_equal(grec["node"], orec["node"])
    assert np.array_equal(grec["uraw"][:, : w.n_ctrl], orec["uraw"][:, : w.n_ctrl])
    assert np.array_equal(grec["k"], orec["k"])
    VALID = 1
    gv = (grec["flags"] & VALID) > 0
    ov = (orec["flags"] & VALID) > 0
    amb = (orec["m_valid"] < TAU) | (orec["m_bin"] < TAU) | (ov & (orec["m_goal"] < TAU))
    differ = ((gv != ov) | (grec["fail_step"] != orec["fail_step"]) |
              (grec["region"] != orec["region"]) | (grec["sub"] != orec["sub"]))
    bad = differ & ~amb
    assert not bad.any(), (
        f"{bad.sum()} non-ambiguous decision mismatches, first keys {np.flatnonzero(bad)[:5]}")
    same = ~differ
    scale = state_scale(w)
    err = np.abs(grec["state"][same] - orec["state"][same]) / scale
    assert err.size == 0 or err.max() <= STATE_TOL, f"state error {err.max():.3g}"
    n_flip = int(differ.sum())
    if before is not None:
        check_downstream(w, ost, orec, gst, grec, amb, before, after, otree, vol)
    if n_flip == 0:
        # all decisions equal: everything downstream is integer and exact
        assert np.array_equal(grec["flags"], orec["flags"]), \
            np.flatnonzero(grec["flags"] != orec["flags"])[:10]
        for key in ("n_valid", "n_accepted", "n_nodes", "goal_node"):
            assert gst[key] == ost[key], (key, gst[key], ost[key])
    if expect_exact:
        assert n_flip == 0
    return n_flip


def compare_trees(w, gt, ot, n_old=None):
    """Exact comparison of two exported trees and decomposition tables;
    states within tolerance."""
    assert gt["n_nodes"] == ot["n_nodes"]
    assert gt["iteration"] == ot["iteration"]
    n = gt["n_nodes"]
    for key in ("parent", "steps", "region", "sub", "in_ve"):
        assert np.array_equal(gt[key][:n], ot[key][:n]), key
    for key in ("n_valid", "n_invalid", "cov", "avail", "thr", "visited"):
        assert np.array_equal(gt[key], ot[key]), (key, np.flatnonzero(gt[key] != ot[key])[:10])
    scale = state_scale(w)
    err = np.abs(gt["state"][:n].astype(np.float64) - ot["state"][:n]) / scale
    assert err.max() <= STATE_TOL, err.max()
    cs = np.asarray(w.u_hi[: w.n_ctrl], np.float64) - np.asarray(w.u_lo[: w.n_ctrl], np.float64)
    cerr = np.abs(gt["ctrl"][:n].astype(np.float64) - ot["ctrl"][:n]) / cs
    assert cerr.max() <= 1e-6, cerr.max()


F_VALID, F_ACCEPTED = 1, 16


def check_downstream(w, ost, orec, gst, grec, amb, before, after, otree, vol):
    """Everything one pass decides after the expand (accept, append, Eq. 3-5,
    node sets, goal), checked against the device's own per-sample records and
    against the oracle wherever no ambiguous sample can have changed the
    outcome.  Samples whose decision lies within TAU of its boundary may flip
    (FP32 against FP64); the checks below hold all the same:

    1. the region counters of the pass equal a recount of the device's own
       per-sample records (every key counted exactly once);
    2. in regions no ambiguous sample reached (on either side) the counters
       equal the oracle's;
    3. a sample that is not ambiguous and whose sub-region no ambiguous
       sample reached has the oracle's flags byte (valid, contender, accept
       draw, representative, appended, goal);
    4. the appended nodes are the device's accepted keys in key order, each
       with its parent (its V_E position's node), duration, region,
       sub-region and end state from its own record, and, for keys of (3),
       the oracle's node within the state tolerance;
    5. visited gains exactly the appended sub-regions; Cov and R_avail
       follow from visited and the node regions;
    6. the thresholds are Eq. 3-5 of the device's own counters, bit for bit
       (the oracle's Eq. 3-5 routine on them);
    7. the next V_E: an old node is in it iff its node-set draw (Philox
       counter (it, v, 0, 2)) is below its region's new threshold; new
       nodes are in it;
    8. the goal node is the smallest new node in the goal ball (checked
       when no new node lies within TAU of its surface)."""
    from oracle import kpo
    S = ost["n_samples"]
    lam = ost["lambda"]
    n0, n1 = int(before["n_nodes"]), int(after["n_nodes"])
    R = len(before["n_valid"])
    per = int(np.prod(w.sub))
    it = int(before["iteration"])
    gflags = grec["flags"][:S]
    gvalid = (gflags & F_VALID) > 0
    greg, gsub = grec["region"][:S], grec["sub"][:S]
    # 1. counters of the pass from the device's own records
    dv = np.bincount(greg[gvalid], minlength=R)
    di = np.bincount(greg[~gvalid], minlength=R)
    cv = after["n_valid"].astype(np.int64) - before["n_valid"].astype(np.int64)
    ci = after["n_invalid"].astype(np.int64) - before["n_invalid"].astype(np.int64)
    assert np.array_equal(cv, dv), np.flatnonzero(cv != dv)[:10]
    assert np.array_equal(ci, di), np.flatnonzero(ci != di)[:10]
    assert int(cv.sum() + ci.sum()) == S
    assert gst["n_valid"] == int(gvalid.sum())
    # 2. untouched regions: the oracle's counters
    touched_r = np.union1d(greg[amb], orec["region"][amb])
    touched_s = np.union1d(gsub[amb], orec["sub"][amb])
    clean_r = np.ones(R, bool)
    clean_r[touched_r] = False
    for key in ("n_valid", "n_invalid"):
        assert np.array_equal(after[key][clean_r], otree[key][clean_r]), key
    # 3. clean samples: the oracle's flags byte
    clean = ~amb & ~np.isin(gsub, touched_s)
    bad = clean & (gflags != orec["flags"][:S])
    assert not bad.any(), np.flatnonzero(bad)[:10]
    # 4. the appended nodes
    gacc = np.flatnonzero(gflags & F_ACCEPTED)
    assert n1 - n0 == len(gacc) == gst["n_accepted"]
    ve = np.flatnonzero(before["in_ve"][:n0])
    ids = n0 + np.arange(len(gacc))
    assert np.array_equal(after["parent"][ids], ve[gacc // lam])
    assert np.array_equal(after["steps"][ids], grec["k"][gacc])
    assert np.array_equal(after["region"][ids], greg[gacc])
    assert np.array_equal(after["sub"][ids], gsub[gacc])
    assert np.array_equal(after["state"][ids].view(np.uint32),
                          grec["state"][gacc].astype(np.float32).view(np.uint32))
    assert np.all(after["in_ve"][ids] == 1)
    oacc = np.flatnonzero(orec["flags"][:S] & F_ACCEPTED)
    common, gi, oi = np.intersect1d(gacc, oacc, return_indices=True)
    keep = clean[common]
    gi, oi = n0 + gi[keep], int(otree["n_nodes"]) - len(oacc) + oi[keep]
    for key in ("parent", "steps", "region", "sub"):
        assert np.array_equal(after[key][gi], otree[key][oi]), key
    scale = state_scale(w)
    err = np.abs(after["state"][gi].astype(np.float64) - otree["state"][oi]) / scale
    assert err.size == 0 or err.max() <= STATE_TOL, err.max()
    # 5. visited, Cov, R_avail
    vis = before["visited"].copy()
    vis[gsub[gacc]] = 1
    assert np.array_equal(after["visited"], vis)
    assert np.array_equal(after["cov"], after["visited"].reshape(-1, per).sum(1))
    av = np.zeros(R, np.uint8)
    av[after["region"][:n1]] = 1
    assert np.array_equal(after["avail"], av)
    # 6. Eq. 3-5 of the device's own tables
    _, _, thr, _ = kpo.eq345_vol(after["n_valid"], after["n_invalid"], after["cov"],
                                 after["avail"], vol, w.delta, w.eps)
    assert np.array_equal(after["thr"], thr), np.flatnonzero(after["thr"] != thr)[:10]
    # 7. the next V_E
    seed = int(w.seed) & 0xFFFFFFFFFFFFFFFF
    ctr = np.zeros((n0, 4), np.uint32)
    ctr[:, 0] = it
    ctr[:, 1] = np.arange(n0)
    ctr[:, 3] = 2
    words = kpo.philox4x32_10_n(ctr, [seed & 0xFFFFFFFF, seed >> 32])
    sel = (words[:, 0].astype(np.uint64) < after["thr"][after["region"][:n0]]).astype(np.uint8)
    assert np.array_equal(after["in_ve"][:n0], sel), np.flatnonzero(after["in_ve"][:n0] != sel)[:10]
    # 8. the goal node
    d = np.linalg.norm(after["state"][n0:n1, :3].astype(np.float64) - w.goal_c, axis=1)
    if len(d) == 0 or np.min(np.abs(d - float(w.goal_r))) >= TAU:
        inside = np.flatnonzero(d <= float(w.goal_r))
        want = n0 + int(inside[0]) if len(inside) else -1
        assert gst["goal_node"] == want, (gst["goal_node"], want)


def check_work(gi0, gi1, ow0, ow1):
    """The device's work counters over one pass whose decisions all matched
    the oracle's equal the oracle's replay count: samples, integrator steps
    and step hulls exactly; broad-phase box tests within 2 % (the device
    places a hull in the grid from FP32 coordinates, the oracle from FP64
    ones, so a hull on a cell face may visit one more or one fewer cell)."""
    for dev, orc in (("n_samples", "samples"), ("n_steps", "steps"), ("n_hull_checks", "hulls")):
        assert gi1[dev] - gi0[dev] == ow1[orc] - ow0[orc], (dev, gi1[dev] - gi0[dev],
                                                           ow1[orc] - ow0[orc])
    db = gi1["n_box_tests"] - gi0["n_box_tests"]
    ob = ow1["box_grid"] - ow0["box_grid"]
    assert abs(db - ob) <= 0.02 * ob + 8, (db, ob)
