"""The seeded input generators produce the workloads they describe: box
counts and sizes, walls with one gap each, start and goal kept clear,
determinism per seed, and the serving mix's ranges (Sec. VI environments,
replaced by synthetic stand-ins of the same kind)."""
import numpy as np
import pytest

from paper_2409_06807_gb300 import workloads as W


def _inside(box, p):
    return bool(np.all(box[:3] <= p) and np.all(p <= box[3:]))


def _ball_clear(boxes, c, r):
    c = np.asarray(c, np.float64)
    for b in boxes.astype(np.float64):
        q = np.clip(c, b[:3], b[3:])
        if np.sum((q - c) ** 2) <= r * r:
            return False
    return True


@pytest.mark.parametrize("make", [W.c1, W.c2, W.c3])
def test_generators_are_seeded(make):
    a, b, c = make(7), make(7), make(8)
    assert np.array_equal(a.boxes, b.boxes)
    assert not np.array_equal(a.boxes, c.boxes)
    assert a.boxes.dtype == np.float32 and a.x_init.dtype == np.float32


def test_c1_random_boxes():
    for seed in range(5):
        w = W.c1(seed)
        assert w.boxes.shape == (16, 6)
        assert np.all(w.boxes[:, :3] >= 0) and np.all(w.boxes[:, 3:] <= 1)
        side = w.boxes[:, 3:] - w.boxes[:, :3]
        assert np.all(side > 0) and np.all(side <= 0.15 + 1e-6)
        assert all(not _inside(b, w.x_init[:3]) for b in w.boxes)
        assert _ball_clear(w.boxes, w.goal_c, float(w.goal_r))
        assert (w.d, w.n_ctrl, w.t_e, w.lambda_max, w.n_regions) == (6, 3, 65536, 32, 512)


def test_c2_forest():
    for seed in range(3):
        w = W.c2(seed)
        assert w.boxes.shape == (200, 6)
        # full-height trunks
        assert np.all(w.boxes[:, 2] == 0) and np.all(w.boxes[:, 5] == 1)
        wid = w.boxes[:, 3:5] - w.boxes[:, 0:2]
        unclipped = np.all((w.boxes[:, 0:2] > 0) & (w.boxes[:, 3:5] < 1), axis=1)
        assert np.all(wid[unclipped] >= 0.02 - 1e-6) and np.all(wid <= 0.04 + 1e-6)
        assert _ball_clear(w.boxes, w.x_init[:3], 0.03)
        assert _ball_clear(w.boxes, w.goal_c, float(w.goal_r))
        assert (w.t_e, w.lambda_max, w.n_regions, w.n_sub_per) == (1 << 20, 64, 4096, 64)


def test_c3_building_has_one_gap_per_wall():
    w = W.c3(3)
    assert w.boxes.shape == (1200, 6)
    pads = [b for b in w.boxes if np.all(b[:3] > 1)]
    assert len(pads) == 3 and all(np.all(p[:3] == p[3:]) for p in pads)
    inside = np.array([b for b in w.boxes if not np.all(b[:3] > 1)])
    assert len(inside) == 3 * 399
    gap = 0.06
    for wx in (0.25, 0.5, 0.75):
        wall = inside[np.isclose((inside[:, 0] + inside[:, 3]) / 2, wx)]
        assert len(wall) == 399
        assert np.allclose(wall[:, 3] - wall[:, 0], 0.02, atol=1e-6)
        # the tiles cover the y-z square but for one gap x gap hole
        area = np.sum((wall[:, 4].astype(np.float64) - wall[:, 1]) * (wall[:, 5] - wall[:, 2]))
        assert area == pytest.approx(1.0 - gap * gap, abs=1e-5)
        # the hole is interior: a point in it meets no tile of this wall,
        # and it is found by scanning a fine y-z lattice
        ys = np.linspace(0.0025, 0.9975, 200)
        y, z = (a.ravel()[:, None] for a in np.meshgrid(ys, ys, indexing="ij"))
        hit = ((wall[:, 1] <= y) & (y <= wall[:, 4]) & (wall[:, 2] <= z) & (z <= wall[:, 5])).any(1)
        assert not hit.all(), "no hole in the wall"
        fy, fz = y[~hit, 0], z[~hit, 0]
        assert fy.max() - fy.min() < gap and fz.max() - fz.min() < gap
        assert 0 < fy.min() and fy.max() < 1 and 0 < fz.min() and fz.max() < 1
    assert w.x_init.shape == (12,) and np.all(w.x_init[3:] == 0)
    assert (w.t_e, w.lambda_max, w.n_regions) == (1 << 22, 128, 16384)


def test_tiny_cases():
    for system in (W.DI, W.DUBINS, W.QUAD):
        w = W.tiny(system, seed=1)
        assert w.boxes.shape == (2, 6) and w.x_init.shape == (W.STATE_DIM[system],)
        assert all(not _inside(b, w.x_init[:3]) for b in w.boxes)
        assert W.tiny(system, n_boxes=0).boxes.shape == (0, 6)


def test_serving_mix_ranges():
    mix = W.serving_mix(n=64, seed=5)
    t = np.array([a for a, _ in mix])
    assert len(mix) == 64 and np.all(np.diff(t) > 0)
    # Poisson at 2,000/s: the mean gap is 0.5 ms, well within a factor 2
    assert 0.25e-3 < t[-1] / 64 < 1e-3
    systems = {w.system for _, w in mix}
    assert systems == {W.DI, W.DUBINS, W.QUAD}
    for _, w in mix:
        assert 16384 <= w.t_e <= 1 << 20
        n_in = int(np.sum(~np.all(w.boxes[:, :3] > 1, axis=1)))
        if w.system == W.QUAD:
            assert 3 <= n_in <= 999
        else:
            assert 10 <= n_in <= 1000
    assert len({w.name for _, w in mix}) == 64
