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


def compare_pass(w, ost, orec, gst, grec, expect_exact=None):
    """Compare one pass.  Returns the number of samples whose decisions
    differ (all of them ambiguous, else AssertionError)."""
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
