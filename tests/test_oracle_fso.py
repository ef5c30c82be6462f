"""Pins of the oracle's free-space-obeying decomposition (Sec. IV-B): a
kd-tree over the workspace split on obstacle faces, whose leaves are the
regions, each with its own volume in Eq. 3."""
import math

import numpy as np

from oracle.kpo import Oracle
from paper_2409_06807_gb300 import workloads as W

ONE_BOX = np.array([[0.25, 0.25, 0.25, 0.75, 0.75, 0.75]], np.float32)

# the seven leaves of a unit workspace around one centred box, worked by
# hand: split on x at 0.25, then y at 0.25, then z at 0.25, then x at 0.75,
# y at 0.75 and z at 0.75 (most distinct faces, lowest axis on a tie, lower
# median), depth first with the side below each plane first
ONE_BOX_LEAVES = [
    ((0.0, 0.0, 0.0), (0.25, 1.0, 1.0)),
    ((0.25, 0.0, 0.0), (1.0, 0.25, 1.0)),
    ((0.25, 0.25, 0.0), (1.0, 1.0, 0.25)),
    ((0.25, 0.25, 0.25), (0.75, 0.75, 0.75)),
    ((0.25, 0.25, 0.75), (0.75, 0.75, 1.0)),
    ((0.25, 0.75, 0.25), (0.75, 1.0, 1.0)),
    ((0.75, 0.25, 0.25), (1.0, 1.0, 1.0)),
]


def _one_box():
    return W.tiny(W.DI, seed=0).with_(boxes=ONE_BOX, fso=True)


def test_one_box_leaves_by_hand():
    o = Oracle(_one_box())
    lo, hi = o.fso_leaves()
    assert o.R == 7 and o.n_sub == 7 * 8
    for r, (elo, ehi) in enumerate(ONE_BOX_LEAVES):
        assert tuple(lo[r]) == elo and tuple(hi[r]) == ehi, r


def test_one_box_binning_by_hand():
    """Points, their leaf, their cell of the 2x2x2 sub-grid inside it and
    the distance to the nearest face that changes either."""
    o = Oracle(_one_box())
    r, s, m = o.bin([0.1, 0.4, 0.3])
    # leaf 0 is [0,.25]x[0,1]x[0,1]: sub cell (0, 0, 0); faces x=.125 (sub)
    # and .25 (leaf), y and z at .5 (sub): nearest 0.025 along x
    assert (r, s) == (0, 0) and math.isclose(m, 0.025, rel_tol=1e-12)
    r, s, m = o.bin([0.4, 0.4, 0.4])
    # the box leaf: sub faces at .5, leaf faces at .25 / .75
    assert (r, s) == (3, 3 * 8) and math.isclose(m, 0.1, rel_tol=1e-12)
    r, s, m = o.bin([0.9, 0.9, 0.3])
    # leaf 6 is [.75,1]x[.25,1]x[.25,1]: x cell 1 (face .875), y cell 1
    # (face .625), z cell 0 (face .625, leaf face .25)
    assert (r, s) == (6, 6 * 8 + 1 + 2) and math.isclose(m, 0.025, rel_tol=1e-12)
    # on a splitting plane the point belongs to the side above it: x = .25
    # is not below the first plane, so it reaches the box leaf, not leaf 0
    r, _, m = o.bin([0.25, 0.6, 0.6])
    assert r == 3 and m == 0.0


def _leaf_of(lo, hi, p):
    inside = np.all((lo <= p) & (p < hi), axis=1)
    assert inside.sum() == 1
    return int(np.flatnonzero(inside)[0])


def test_leaves_tile_and_obey_free_space():
    """On the forest and building layouts: the leaves tile the workspace
    (volumes sum to it, every point lies in exactly one), and no obstacle
    face crosses a leaf, so each leaf is inside an obstacle or meets none."""
    for w in (W.c2(0), W.c3(0), W.c1(1)):
        o = Oracle(w.with_(fso=True))
        lo, hi = o.fso_leaves()
        assert o.R == len(lo) > 1
        ws = np.prod(w.ws_hi.astype(np.float64) - w.ws_lo)
        assert math.isclose(math.fsum(np.prod(hi - lo, axis=1)), ws, rel_tol=1e-12)
        b = np.asarray(w.boxes, np.float64)
        for r in range(len(lo)):
            meets = np.all((b[:, :3] < hi[r]) & (b[:, 3:] > lo[r]), axis=1)
            contains = np.all((b[:, :3] <= lo[r]) & (b[:, 3:] >= hi[r]), axis=1)
            assert np.all(contains[meets]), r
        rng = np.random.default_rng(5)
        pts = w.ws_lo + rng.random((300, 3)) * (w.ws_hi - w.ws_lo)
        for p in pts:
            _leaf_of(lo, hi, p)


def test_binning_matches_brute_force():
    """Region = the leaf holding the point (found by scanning every leaf),
    sub = the sub-grid cell inside it, margin = the nearest face that is not
    on the workspace boundary: a leaf face or a sub-grid face."""
    w = W.c2(0).with_(fso=True)
    o = Oracle(w)
    lo, hi = o.fso_leaves()
    wlo = w.ws_lo.astype(np.float64)
    whi = w.ws_hi.astype(np.float64)
    n = np.asarray(w.sub)
    rng = np.random.default_rng(9)
    for p in wlo + rng.random((400, 3)) * (whi - wlo):
        r = _leaf_of(lo, hi, p)
        ext = hi[r] - lo[r]
        t = (p - lo[r]) * n / ext
        fine = np.minimum(np.floor(t).astype(int), n - 1)
        k = fine[0] + n[0] * (fine[1] + n[1] * fine[2])
        m = math.inf
        for a in range(3):
            faces = [lo[r][a] + f * ext[a] / n[a] for f in range(1, n[a])]
            if lo[r][a] > wlo[a]:
                faces.append(lo[r][a])
            if hi[r][a] < whi[a]:
                faces.append(hi[r][a])
            for f in faces:
                m = min(m, abs(p[a] - f) / (whi[a] - wlo[a]))
        gr, gs, gm = o.bin(p)
        assert (gr, gs) == (r, r * o.n_sub // o.R + k)
        assert math.isclose(gm, m, rel_tol=1e-9, abs_tol=1e-15)


def test_no_obstacles_is_the_one_cell_grid():
    """Without obstacles the kd-tree is one leaf, the workspace; the whole
    planner must then run exactly as with a 1x1x1 grid (same volume, same
    sub-grid), pass for pass."""
    for system in (W.DI, W.DUBINS):
        base = W.tiny(system, seed=1, n_boxes=0, t_e=3000, lambda_max=8)
        a = Oracle(base.with_(fso=True))
        b = Oracle(base.with_(grid=(1, 1, 1)))
        assert a.R == b.R == 1
        a.reset()
        b.reset()
        for _ in range(6):
            sa, _, _ = a.iterate()
            sb, _, _ = b.iterate()
            assert sa == sb
            ea, eb = a.export(), b.export()
            for key in ea:
                assert np.array_equal(ea[key], eb[key]), key


def test_eq3_per_region_volume(kpo):
    """Two regions with equal counts, one twice the other's volume: FreeVol
    doubles and Score (Eq. 4, FreeVol to the fourth) grows sixteen-fold, so
    the normalised scores of Eq. 5 are 1/17 and 16/17."""
    eps = 0.01
    score, p, thr, s = kpo.eq345_vol([4, 4], [2, 2], [3, 3], [1, 1], [0.125, 0.25], 1.0, eps)
    assert score[1] == 16.0 * score[0]
    assert math.isclose(p[0], 1 / 17 + eps, rel_tol=1e-15)
    assert math.isclose(p[1], 16 / 17 + eps, rel_tol=1e-15)


def test_planner_scores_use_leaf_volumes(kpo):
    """The planner's region scores after a few passes are Eq. 3-5 over its
    counts with each leaf's own volume (not one volume for all)."""
    w = W.c2(0).with_(fso=True, t_e=1 << 16)
    o = Oracle(w)
    o.reset()
    o.run(3)
    lo, hi = o.fso_leaves()
    vol = (hi[:, 0] - lo[:, 0]) * (hi[:, 1] - lo[:, 1]) * (hi[:, 2] - lo[:, 2])
    e = o.export()
    score, p, s = o.estimates()
    es, ep, _, _ = kpo.eq345_vol(e["n_valid"], e["n_invalid"], e["cov"], e["avail"], vol,
                                 w.delta, w.eps)
    assert np.count_nonzero(e["avail"]) > 10
    assert np.array_equal(score, es) and np.array_equal(p, ep)
    # the available leaves differ in volume, so one volume for all fails
    a = np.flatnonzero(e["avail"])
    assert len(set(np.round(vol[a], 12))) > 1


def test_learned_features_have_no_grid_neighbours():
    """The neighbour entries of the node features are a position-grid notion;
    under the kd-tree they stay zero while the rest is filled."""
    w = W.tiny(W.DI, seed=0, t_e=2000, lambda_max=8).with_(boxes=ONE_BOX, fso=True)
    o = Oracle(w)
    o.reset()
    o.run(3)
    for v in range(min(o.export()["parent"].size, 40)):
        f = o.features(v)
        assert np.all(f[14:20] == 0.0)
        assert f[13] > 0.0


def _many_small_boxes(n):
    return W.random_boxes(5, n, side=(0.01, 0.03),
                          keep_clear=[((0.1, 0.1, 0.1), 0.02), ((0.9, 0.9, 0.9), 0.06)])


def test_leaf_capacity():
    """1,000 small random boxes give a tree within the 16,384-leaf capacity
    (it still tiles W); 2,000 exceed it and the oracle refuses the set."""
    import pytest
    w = W.c1(0).with_(boxes=_many_small_boxes(1000), fso=True)
    o = Oracle(w)
    lo, hi = o.fso_leaves()
    assert 1000 < o.R <= 16384
    assert math.isclose(math.fsum(np.prod(hi - lo, axis=1)), 1.0, rel_tol=1e-12)
    with pytest.raises(ValueError):
        Oracle(w.with_(boxes=_many_small_boxes(2000)))
