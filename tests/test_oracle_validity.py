"""Pins of the oracle's validity check (Sec. II valid set, Algorithm 2) and
its region binning (Sec. III decomposition)."""
import numpy as np

from oracle.kpo import Oracle
from paper_2409_06807_gb300 import workloads as W

BOX = np.array([[0.4, 0.4, 0.4, 0.6, 0.6, 0.6]], np.float32)


def _di(**kw):
    return Oracle(W.tiny(W.DI, n_boxes=0).with_(boxes=BOX, **kw))


def _state(p, v=(0, 0, 0)):
    return np.array([*p, *v], np.float64)


def test_touching_a_face_collides():
    """Obstacles are closed sets: a segment ending exactly on a face hits."""
    o = _di()
    face = float(BOX[0, 0])  # the float32 face value the planner sees
    ok, m = o.step_valid(_state((0.3, 0.5, 0.5)), _state((face, 0.5, 0.5)))
    assert not ok and m == 0.0
    ok, m = o.step_valid(_state((0.3, 0.5, 0.5)),
                         _state((np.nextafter(face, 0.0), 0.5, 0.5)))
    assert ok and m > 0.0


def test_clear_segment_margin():
    o = _di()
    ok, m = o.step_valid(_state((0.1, 0.5, 0.5)), _state((0.35, 0.5, 0.5)))
    assert ok and abs(m - (float(BOX[0, 0]) - 0.35)) < 1e-15


def test_corner_cut_is_conservative():
    """A diagonal segment that passes the corner without touching the box
    still has an axis-aligned hull that overlaps it: invalid (coarse phase)."""
    o = _di()
    a, b = _state((0.30, 0.58, 0.5)), _state((0.42, 0.70, 0.5))
    # the straight segment itself stays outside the box:
    t = np.linspace(0, 1, 10001)[:, None]
    pts = a[None, :3] * (1 - t) + b[None, :3] * t
    inside = np.all((pts >= BOX[0, :3]) & (pts <= BOX[0, 3:]), axis=1)
    assert not inside.any()
    ok, _ = o.step_valid(a, b)
    assert not ok


def test_state_bounds():
    o = _di()
    ok, m = o.step_valid(_state((0.1, 0.1, 0.1)), _state((0.1, 0.1, 0.1), (0.31, 0, 0)))
    assert not ok and m > 0
    ok, m = o.step_valid(_state((0.1, 0.1, 0.1)), _state((0.1, 0.1, 0.1), (0.3, 0, 0)))
    assert ok  # closed bound
    ok, _ = o.step_valid(_state((0.9, 0.1, 0.1)), _state((1.0001, 0.1, 0.1)))
    assert not ok  # leaving the workspace
    ok, _ = o.step_valid(_state((0.1, 0.1, 0.1)), _state((0.1, 0.1, np.nan)))
    assert not ok  # NaN is never valid


def test_state_box_is_closed_on_both_sides():
    """The state box is a closed set: a state exactly on a bound (the float32
    value the planner holds) is valid, the next double outwards is not."""
    w = W.tiny(W.DI, n_boxes=0)
    o = Oracle(w)
    base = _state((0.5, 0.5, 0.5))
    for i in range(6):
        for bound, out in ((float(w.x_lo[i]), -1.0), (float(w.x_hi[i]), 1.0)):
            on = base.copy()
            on[i] = bound
            ok, _ = o.step_valid(base, on)
            assert ok, (i, bound)
            off = on.copy()
            off[i] = np.nextafter(bound, bound + out)
            ok, _ = o.step_valid(base, off)
            assert not ok, (i, bound)


def test_axis_aligned_segments_match_dense_sampling():
    """For a segment along one axis the hull is the segment itself, so the
    check must agree with dense point sampling (brute force)."""
    rng = np.random.default_rng(3)
    o = _di()
    for _ in range(400):
        a = rng.uniform(0.2, 0.8, 3)
        b = a.copy()
        ax = rng.integers(3)
        b[ax] = rng.uniform(0.2, 0.8)
        ok, m = o.step_valid(_state(a), _state(b))
        if abs(m) < 1e-3:
            continue
        t = np.linspace(0, 1, 2001)[:, None]
        pts = a[None] * (1 - t) + b[None] * t
        hit = np.any(np.all((pts >= BOX[0, :3]) & (pts <= BOX[0, 3:]), axis=1))
        assert ok == (not hit)


def test_hull_valid_implies_dense_valid_di():
    """Euler steps are straight segments inside their hull: a hull-valid
    double-integrator edge is valid at every dense sample (exactly)."""
    w = W.c1(3)
    o = Oracle(w)
    rng = np.random.default_rng(5)
    checked = 0
    while checked < 150:
        x0 = np.concatenate([rng.uniform(0, 1, 3), rng.uniform(-0.3, 0.3, 3)])
        if not o.step_valid(x0, x0)[0]:
            continue
        u = rng.uniform(-0.5, 0.5, 3)
        k = int(rng.integers(1, 11))
        x, valid = x0.copy(), True
        from oracle.kpo import step
        for _ in range(k):
            nx = step(w, x, u)
            valid, _ = o.step_valid(x, nx)
            x = nx
            if not valid:
                break
        if valid:
            depth, xe = o.dense_check(x0, u, k, 100)
            assert depth <= 0.0
            np.testing.assert_allclose(xe, x, atol=1e-14)
            checked += 1


def test_hull_valid_implies_dense_valid_dubins():
    """RK4 sub-paths bend slightly between steps: dense violations of a
    hull-valid Dubins edge stay below the curvature bound (1e-4)."""
    w = W.c2(1)
    o = Oracle(w)
    rng = np.random.default_rng(6)
    from oracle.kpo import step
    checked = 0
    while checked < 60:
        x0 = np.array([*rng.uniform(0, 1, 3), rng.uniform(-3, 3),
                       rng.uniform(-0.5, 0.5), rng.uniform(0.05, 0.2)])
        if not o.step_valid(x0, x0)[0]:
            continue
        u = rng.uniform([-1, -0.5, -0.1], [1, 0.5, 0.1])
        k = int(rng.integers(1, 21))
        x, valid = x0.copy(), True
        for _ in range(k):
            nx = step(w, x, u)
            valid, _ = o.step_valid(x, nx)
            x = nx
            if not valid:
                break
        if valid:
            depth, _ = o.dense_check(x0, u, k, 100)
            assert depth <= 1e-4
            checked += 1


def test_binning_cell_centres():
    """Every fine-cell centre of a 2^3 x 2^3 decomposition lands in the
    region and sub-region boxes that contain it; the map is a bijection."""
    w = W.tiny(W.DI, n_boxes=0)
    o = Oracle(w)
    seen = set()
    for fx in range(4):
        for fy in range(4):
            for fz in range(4):
                c = (np.array([fx, fy, fz]) + 0.5) / 4
                r, s, m = o.bin(np.concatenate([c, [0, 0, 0]]))
                assert abs(m - 0.125) < 1e-15  # half a fine cell from a face
                ix, iy, iz = r % 2, (r // 2) % 2, r // 4
                lo = np.array([ix, iy, iz]) / 2
                assert np.all(lo <= c) and np.all(c < lo + 0.5)
                k = s - r * 8
                jx, jy, jz = k % 2, (k // 2) % 2, k // 4
                slo = lo + np.array([jx, jy, jz]) / 4
                assert np.all(slo <= c) and np.all(c < slo + 0.25)
                seen.add(s)
    assert seen == set(range(64))


def test_binning_clamps():
    o = Oracle(W.tiny(W.DI, n_boxes=0))
    r_hi, s_hi, _ = o.bin(np.array([1.0, 1.0, 1.0, 0, 0, 0]))
    assert r_hi == 7 and s_hi == 63        # the hi face belongs to the last cell
    r_out, s_out, _ = o.bin(np.array([1.7, -0.2, 1.0, 0, 0, 0]))
    assert r_out == 1 + 4 and s_out == 5 * 8 + 1 + 4
    r_nan, s_nan, m = o.bin(np.array([np.nan, 0.1, 0.1, 0, 0, 0]))
    assert r_nan == 0 and s_nan == 0 and m == 0.0


def test_speed_bins():
    """Quadrotor regions append 4 speed bins over [0, 0.5] (clamped)."""
    w = W.c3(0)
    o = Oracle(w)
    x = np.zeros(12)
    x[:3] = 0.01
    for speed, expect in ((0.0, 0), (0.1, 0), (0.13, 1), (0.3, 2), (0.45, 3), (0.9, 3)):
        x[6:9] = (speed, 0, 0)
        r, _, _ = o.bin(x)
        assert r // 4096 == expect


def test_state_grid_binning_by_hand():
    """A grid over the Dubins state space (Sec. VI: grid dimension equal to
    the state dimension): 2^3 position cells x 4 heading cells over
    [-pi, pi) (the heading is wrapped) x 2 pitch cells over [-pi/6, pi/6] x
    2 speed cells over [0.05, 0.2].  Cell centres land in the cell built by
    hand from the mixed radix (position fastest, then heading, pitch,
    speed); region count 8 * 16."""
    sg = [0] * 12
    sg[3], sg[4], sg[5] = 4, 2, 2
    w = W.tiny(W.DUBINS, n_boxes=0, state_grid=tuple(sg))
    o = Oracle(w)
    assert o.R == 8 * 16
    th = np.pi / 6
    seen = set()
    for cpos in range(8):
        # centre of the first fine cell of position region cpos (2 x 2 x 2
        # fine cells per region)
        p = (2 * np.array([cpos % 2, (cpos // 2) % 2, cpos // 4]) + 0.5) / 4
        for ch in range(4):
            psi = -np.pi + (ch + 0.5) * (2 * np.pi / 4)
            for cp in range(2):
                pitch = -th + (cp + 0.5) * th
                for cv in range(2):
                    v = 0.05 + (cv + 0.5) * 0.075
                    r, s, m = o.bin(np.array([*p, psi, pitch, v]))
                    expect = cpos + 8 * (ch + 4 * (cp + 2 * cv))
                    assert r == expect
                    assert abs(m - 0.125) < 1e-12  # half a fine cell, half a heading cell
                    seen.add(r)
    assert seen == set(range(128))


def test_state_grid_wraps_and_clamps():
    sg = [0] * 12
    sg[3], sg[4], sg[5] = 4, 2, 2
    o = Oracle(W.tiny(W.DUBINS, n_boxes=0, state_grid=tuple(sg)))
    base = np.array([0.1, 0.1, 0.1, 0.0, 0.0, 0.1])
    # heading pi + 0.1 wraps to -pi + 0.1 (cell 0); -pi - 0.1 to pi - 0.1 (cell 3)
    for psi, cell in ((np.pi + 0.1, 0), (-np.pi - 0.1, 3), (3 * np.pi + 0.2, 0), (0.01, 2)):
        x = base.copy()
        x[3] = psi
        r, _, _ = o.bin(x)
        assert (r // 8) % 4 == cell, (psi, r)
    # the wrap point is a face of the heading cells
    x = base.copy()
    x[3] = np.pi - 1e-6
    _, _, m = o.bin(x)
    assert m < 1e-6
    # pitch and speed clamp to their end cells outside the box
    x = base.copy()
    x[4], x[5] = 1.0, 0.5
    r, _, _ = o.bin(x)
    assert (r // 32) % 2 == 1 and r // 64 == 1
    x[4], x[5] = -1.0, 0.0
    r, _, _ = o.bin(x)
    assert (r // 32) % 2 == 0 and r // 64 == 0
