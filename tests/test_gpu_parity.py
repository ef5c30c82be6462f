"""CUDA planner vs the FP64 oracle, element by element, through the C ABI.

Every input is a seeded synthetic workload (or a tree state the oracle grew
from one); nothing the device computes feeds the oracle."""
import numpy as np
import pytest

from oracle import kpo
from oracle.kpo import Oracle
from paper_2409_06807_gb300 import workloads as W
from parity_util import check_work, compare_pass, compare_trees, state_scale

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import os
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2409_06807_gb300.build import build_planner
    from paper_2409_06807_gb300 import planner
    if os.environ.get("KP_TEST_BOUNDS_CHECKED") == "1":
        # tests/test_gpu_checked.py reruns suites of this file on the
        # bounds-checked build, in a process of their own
        planner.use_library(build_planner(check=True))
        assert planner.lib().kp_bounds_checked() == 1
    else:
        build_planner()
    return planner


def _as_input(t):
    """A device tree as oracle input (float32 rows, as the device holds them)."""
    t = dict(t)
    t["state"] = np.asarray(t["state"], np.float32)
    t["ctrl"] = np.asarray(t["ctrl"], np.float32)
    return t


def lockstep(P, w, n_iters, log_cap=None, grid=None):
    """Both implementations from the same root; every pass is compared.
    A pass whose decisions all agree must give the oracle's tree exactly;
    after a pass in which ambiguous samples (decisions within 1e-4 of their
    boundary) flipped, everything downstream is checked against the device's
    own records and the oracle's unaffected part (check_downstream), and the
    oracle continues from the device's tree: the tree is an input of the
    next pass, never a decision.  'grid' caps the launch at that many blocks
    (the key-batch counter and lane refills then run on every pass).
    Returns (passes with no flip, passes run, flipped samples, samples, info)."""
    g = P.Planner(w)
    if grid:
        g.set_grid_limit(grid)
    o = Oracle(w)
    bp = g.info()["bp_grid"]
    o.set_work_grid(bp)
    vol = o.region_volumes()
    assert g.reset() == P.OK and o.reset() == kpo.RUNNING
    g.enable_log(log_cap or w.t_e)
    exact = flips_total = samples = 0
    before = g.export_tree()
    i = -1
    for i in range(n_iters):
        gi0, ow0 = g.info(), o.work()
        status, ost, orec = o.iterate(records=True)
        gstats = g.expand_step(1)
        if status == kpo.FULL:
            assert gstats == [] and g.info()["state"] == 2
            break
        assert len(gstats) == 1
        grec = g.read_log(ost["n_samples"])
        after = g.export_tree()
        ot = o.export()
        flips = compare_pass(w, ost, orec, gstats[0], grec, before=before, after=after,
                             otree=ot, vol=vol)
        flips_total += flips
        samples += ost["n_samples"]
        if flips == 0:
            compare_trees(w, after, ot)
            check_work(gi0, g.info(), ow0, o.work())
            exact += 1
        else:
            o = Oracle(w)
            o.set_work_grid(bp)
            o.import_(_as_input(after))
        before = after
        if gstats[0]["goal_node"] >= 0:
            assert g.info()["state"] == 1
            break
    info = g.info()
    # every key of every pass was counted exactly once in a region counter
    assert int(before["n_valid"].sum() + before["n_invalid"].sum()) == info["n_samples"]
    return exact, i + 1, flips_total, samples, info


@pytest.mark.parametrize("system", [W.DI, W.DUBINS, W.QUAD])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lockstep_tiny(P, system, seed):
    w = W.tiny(system, seed=seed, t_e=2000, lambda_max=8)
    exact, ran, flips, n, _ = lockstep(P, w, 12)
    assert exact >= min(ran, 3)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_lockstep_c1(P, seed):
    """Double integrator, 16 boxes, 8^3 x 4^3 decomposition, lambda 32,
    t_e 65,536: passes of 32 .. ~60,000 samples (many tiles, ragged), in the
    full launch shape; every pass compared."""
    w = W.c1(seed)
    exact, ran, flips, n, _ = lockstep(P, w, 12)
    # FP32 and FP64 disagree on about 1e-5 of the samples (all within 1e-4
    # of a boundary), so with 30-60 k samples a pass, some passes carry a
    # flip; those passes are checked by check_downstream instead
    assert exact >= ran // 2, (exact, ran, flips, n)
    assert flips <= 1e-4 * n


@pytest.mark.parametrize("grid", [1, 2, 3])
@pytest.mark.parametrize("seed", [0, 1])
def test_lockstep_c1_refill_path(P, grid, seed):
    """The same double-integrator queries on 1-3 blocks: every lane runs
    hundreds of keys of a large pass, taken in batches from the grid-wide
    key counter and started as lanes finish (the path every full-size pass
    takes).  The device counts those batches and refills; both must be
    non-zero, and every pass must match the oracle as in the full launch."""
    w = W.c1(seed)
    exact, ran, flips, n, info = lockstep(P, w, 12, grid=grid)
    assert info["grid_blocks"] == grid
    assert info["n_key_batches"] > 0 and info["n_lane_refills"] > 0, info
    # at most one first key per lane and pass: the rest were refills
    assert info["n_lane_refills"] >= n - ran * grid * 256
    assert exact >= ran // 2, (exact, ran, flips, n)
    assert flips <= 1e-4 * n


@pytest.mark.parametrize("system", [W.DUBINS, W.QUAD])
def test_lockstep_refill_path_rk4(P, system):
    """The RK4 systems on one block, passes of thousands of samples."""
    w = W.tiny(system, seed=0, t_e=20000, lambda_max=32)
    exact, ran, flips, n, info = lockstep(P, w, 8, grid=1)
    assert info["n_key_batches"] > 0 and info["n_lane_refills"] > 0, info
    assert exact >= min(ran, 4), (exact, ran, flips, n)


def frontier(P, w, grow, n_pass=1, all_in_ve=False, grid=None):
    """The oracle grows a tree for 'grow' passes; its state (rounded to
    float32) is loaded into the device planner and into a fresh oracle, and
    both run n_pass passes, compared as in lockstep.  all_in_ve puts every
    node of the grown tree in V_E (a larger frontier; an input like the
    tree itself)."""
    src = Oracle(w)
    src.reset()
    for _ in range(grow):
        src.iterate()
    t = _as_input(src.export())
    if all_in_ve:
        t["in_ve"][:] = 1
    o = Oracle(w)
    g = P.Planner(w)
    bp = g.info()["bp_grid"]
    o.set_work_grid(bp)
    o.import_(t)
    vol = o.region_volumes()
    if grid:
        g.set_grid_limit(grid)
    g.import_tree(t)
    start = g.export_tree()
    for key in ("parent", "region", "sub", "in_ve", "n_valid", "n_invalid", "thr", "visited"):
        assert np.array_equal(start[key], t[key]), key
    assert np.array_equal(start["cov"], t["cov"]) and np.array_equal(start["avail"], t["avail"])
    g.enable_log(w.t_e)
    flips_total = 0
    before = start
    for _ in range(n_pass):
        gi0, ow0 = g.info(), o.work()
        status, ost, orec = o.iterate(records=True)
        gs = g.expand_step(1)
        assert len(gs) == 1
        after = g.export_tree()
        ot = o.export()
        flips = compare_pass(w, ost, orec, gs[0], g.read_log(ost["n_samples"]), before=before,
                             after=after, otree=ot, vol=vol)
        flips_total += flips
        if flips == 0:
            compare_trees(w, after, ot)
            check_work(gi0, g.info(), ow0, o.work())
        else:
            o = Oracle(w)
            o.set_work_grid(bp)
            o.import_(_as_input(after))
        before = after
        if status != kpo.RUNNING or gs[0]["goal_node"] >= 0:
            break
    return flips_total, ost


def test_frontier_c2_full_shape_refill(P):
    """The Dubins forest in the full launch shape with a frontier of every
    node of the oracle's 4-pass tree (16,746 nodes, lambda 61 by Eq. 6:
    about 1.02 M samples, more than 8 keys per lane of the 116,736-lane
    launch): the pass the benchmark's large passes take, lane refills and
    key batches included, compared sample by sample."""
    w = W.c2(0)
    flips, ost = frontier(P, w, grow=4, all_in_ve=True)
    g_lanes = P.Planner(w).info()["grid_blocks"] * 256
    assert ost["n_samples"] >= 4 * g_lanes, (ost["n_samples"], g_lanes)
    assert flips <= 1e-4 * ost["n_samples"]


def test_frontier_c2_dubins(P):
    """Dubins airplane, 200-trunk forest, 16^3 x 4^3, lambda 64, t_e 2^20:
    one pass over the oracle's 3-pass tree (~10^5 samples)."""
    flips, ost = frontier(P, W.c2(0), grow=2)
    assert ost["n_samples"] > 10000
    assert flips <= 2


def test_frontier_c3_quadrotor(P):
    """Quadrotor, 1,200-box building, 16^3 x 4 speed bins x 4^3, lambda
    128, t_e 2^22: one pass over the oracle's 1-pass tree (~1.6e4 samples)."""
    flips, ost = frontier(P, W.c3(0), grow=1)
    assert ost["n_samples"] > 10000
    assert flips <= 2


def test_frontier_empty_v_e(P):
    """A pass with V_E empty draws no sample but still re-selects nodes."""
    w = W.c1(0)
    src = Oracle(w)
    src.reset()
    src.run(3)
    t = src.export()
    t["in_ve"][:] = 0
    o = Oracle(w)
    o.import_(t)
    g = P.Planner(w)
    g.import_tree(t)
    status, ost, _ = o.iterate()
    gs = g.expand_step(1)
    assert ost["n_samples"] == 0 and gs[0]["n_samples"] == 0
    compare_trees(w, g.export_tree(), o.export())


def _revalidate(w, traj, x_init, tol=1e-4):
    """Re-propagate every edge in FP64 from the returned parent state:
    child state within tol, dense check within tol, goal reached."""
    o = Oracle(w)
    scale = state_scale(w)
    prev = np.asarray(x_init, np.float64)
    for e in range(len(traj["steps"])):
        u = traj["ctrls"][e].astype(np.float64)
        depth, x_end = o.dense_check(prev, u, int(traj["steps"][e]), 100)
        assert depth <= tol, f"edge {e} penetrates by {depth}"
        err = np.abs(x_end - traj["states"][e]) / scale
        assert err.max() <= tol, f"edge {e} re-propagation error {err.max()}"
        prev = traj["states"][e].astype(np.float64)
    end = traj["states"][-1][:3].astype(np.float64)
    assert np.linalg.norm(end - w.goal_c) <= float(w.goal_r) * (1 + 1e-6)


@pytest.mark.parametrize("seed", range(4))
def test_plan_c1_revalidated(P, seed):
    w = W.c1(seed)
    g = P.Planner(w)
    st, traj = g.plan(max_iters=200)
    assert st == P.OK and len(traj["steps"]) > 0
    _revalidate(w, traj, w.x_init)
    _tree_invariants(w, g.export_tree(), info=g.info())


@pytest.mark.parametrize("seed", range(2))
def test_plan_c2_full_size(P, seed):
    """Full-size Dubins forest query, the configuration the benchmark times:
    the returned trajectory is re-validated edge by edge by the oracle, and
    tree-wide invariants hold."""
    w = W.c2(seed)
    g = P.Planner(w)
    st, traj = g.plan(max_iters=200)
    assert st == P.OK
    _revalidate(w, traj, w.x_init)
    info = g.info()
    assert info["n_key_batches"] > 0 and info["n_lane_refills"] > 0, info
    _tree_invariants(w, g.export_tree(), sample_edges=300, info=info)


def test_trajectory_extraction_both_paths(P):
    """The root-to-goal chain is written after the passes by one block:
    one thread walks the parent links once and keeps the node ids in shared
    memory, then the block writes the rows; a chain longer than that room
    goes down a one-thread second walk.  The rows equal the chain read from
    the exported tree, and with the room capped below the chain's length
    (the second walk) the same query gives the same bits."""
    w = W.c2(1)
    g = P.Planner(w)
    st, traj = g.plan(max_iters=200)
    assert st == P.OK
    n = len(traj["steps"])
    assert n >= 3
    t = g.export_tree()
    chain, v = [], g.info()["goal_node"]
    while v > 0:
        chain.append(v)
        v = t["parent"][v]
    chain = chain[::-1]
    assert len(chain) == n
    assert np.array_equal(traj["states"], t["state"][chain])
    assert np.array_equal(traj["ctrls"], t["ctrl"][chain])
    assert np.array_equal(traj["steps"], t["steps"][chain])
    for cap in (1, n - 1, n):
        g.set_extract_ids(cap)
        st2, traj2 = g.plan(max_iters=200)
        assert st2 == P.OK
        for k in ("states", "ctrls", "steps"):
            assert np.array_equal(traj2[k], traj[k]), (cap, k)
    g.set_extract_ids(0)
    with pytest.raises(P.KpError):
        g.set_extract_ids(-1)


def _tree_invariants(w, t, sample_edges=0, info=None):
    n = t["n_nodes"]
    if info is not None:
        # every sample of every pass since the reset was counted exactly once
        assert int(t["n_valid"].sum() + t["n_invalid"].sum()) == info["n_samples"]
    assert 1 <= n <= w.t_e
    assert t["parent"][0] == -1 and np.all(t["parent"][1:n] < np.arange(1, n))
    assert np.all(t["parent"][1:n] >= 0)
    per = w.n_sub_per
    assert np.array_equal(t["cov"], t["visited"].reshape(-1, per).sum(1))
    av = np.zeros_like(t["avail"])
    av[t["region"][:n]] = 1
    assert np.array_equal(t["avail"], av)
    assert np.all(t["visited"][t["sub"][:n]] == 1)
    assert np.all(t["sub"][:n] // per == t["region"][:n])
    thr = t["thr"].astype(np.float64) / 2 ** 32
    assert np.all(thr[t["avail"] == 0] == 1.0)
    assert np.all(thr[t["avail"] == 1] >= w.eps - 2 ** -32)
    if sample_edges:
        o = Oracle(w)
        rng = np.random.default_rng(0)
        scale = state_scale(w)
        for v in rng.integers(1, n, size=min(sample_edges, n - 1)):
            p = t["parent"][v]
            traj = kpo.propagate(w, t["state"][p].astype(np.float64),
                                 t["ctrl"][v].astype(np.float64), int(t["steps"][v]))
            err = np.abs(traj[-1] - t["state"][v]) / scale
            assert err.max() <= 1e-4
            r, s, m = o.bin(traj[-1])
            if m > 1e-4:
                assert r == t["region"][v] and s == t["sub"][v]


def test_tree_full_stops(P):
    w = W.tiny(W.DI, seed=1, t_e=40, goal_r=np.float32(0.0))
    g = P.Planner(w)
    st, _ = g.plan(max_iters=100)
    assert st == P.NO_SOLUTION
    info = g.info()
    assert info["state"] == 2 and info["n_nodes"] <= 40
    o = Oracle(w)
    o.reset()
    status, _ = o.run(100)
    assert status == kpo.FULL


def test_root_cases(P):
    w = W.tiny(W.DI)
    g = P.Planner(w)
    st, traj = g.plan(max_iters=5, x_init=w.x_init,
                      goal=P.goal_struct(w.with_(goal_c=w.x_init[:3].copy())))
    assert st == P.OK and len(traj["steps"]) == 0
    bad = w.x_init.copy()
    bad[3] = 5.0
    with pytest.raises(P.KpError) as e:
        g.reset(x_init=bad)
    assert e.value.status == P.ERR_ARG
    assert g.reset() == P.OK  # the context is still usable


def test_no_obstacles_and_obstacle_swap(P):
    w = W.c1(0)
    g = P.Planner(w.with_(boxes=np.zeros((0, 6), np.float32)), box_capacity=16)
    st, traj = g.plan(max_iters=100)
    assert st == P.OK
    g.set_obstacles(w.boxes)
    g.w = w
    st, traj = g.plan(max_iters=100)
    assert st == P.OK
    _revalidate(w, traj, w.x_init)


def test_consecutive_queries_start_clean(P):
    """A query's launch clears the tables and writes the root itself: a
    query planned on a context that just planned other layouts (other trees
    and obstacles) gives the same bits as on a fresh context.  The context
    keeps the random key it was created with, so the fresh contexts take
    that key too."""
    seq = [W.c2(5), W.c2(6).with_(seed=5), W.c2(7).with_(seed=5)]
    g = P.Planner(seq[0])
    used = []
    for w in seq:
        g.set_obstacles(w.boxes)
        g.w = w
        st, traj = g.plan(max_iters=200)
        used.append((st, traj, g.info()))
    for w, (st, traj, info) in zip(seq, used):
        f = P.Planner(w)
        st2, traj2 = f.plan(max_iters=200)
        info2 = f.info()
        assert st == st2
        for k in ("states", "ctrls", "steps"):
            assert np.array_equal(traj[k], traj2[k]), k
        for k in ("n_nodes", "n_samples", "n_steps", "iteration"):
            assert info[k] == info2[k], k
        f.close()


def test_budget_iterations(P):
    w = W.c2(0)
    g = P.Planner(w)
    st, _ = g.plan(max_iters=2)
    assert st == P.NO_SOLUTION and g.info()["iteration"] == 2


def test_bounded_wait_reports_timeout(P):
    """A device wait on a flag nothing sets ends after the wait limit with
    KP_ERR_TIMEOUT; the context is then poisoned, other contexts are not."""
    w = W.tiny(W.DI)
    g = P.Planner(w)
    g.set_wait_limit(2_000_000)  # 2 ms
    assert g.selftest_wait_timeout() == P.ERR_TIMEOUT
    with pytest.raises(P.KpError) as e:
        g.reset()
    assert e.value.status == P.ERR_STATE
    h = P.Planner(w)
    assert h.reset() == P.OK


def test_broad_phase_coarsens_for_large_boxes(P):
    """Many boxes spanning most of the workspace overflow the finest
    broad-phase grid; the planner coarsens it and the verdicts still match
    the oracle's test of every box."""
    rng = np.random.default_rng(7)
    n = 600
    lo = rng.uniform(0.0, 0.45, (n, 3)).astype(np.float32)
    hi = (lo + rng.uniform(0.3, 0.5, (n, 3))).astype(np.float32)
    boxes = np.concatenate([lo, hi], 1)
    w = W.tiny(W.DI, seed=3, t_e=3000, lambda_max=16)
    p0 = w.x_init[:3]
    keep = ~np.all((boxes[:, :3] <= p0 + 0.06) & (boxes[:, 3:] >= p0 - 0.06), axis=1)
    w = w.with_(boxes=boxes[keep][:400])
    g = P.Planner(w)
    g.reset()
    assert g.info()["bp_cells"] < 4096
    exact, ran, flips, n, _ = lockstep(P, w, 6)
    assert exact >= min(ran, 2)


def test_broad_phase_grid_shape_follows_the_obstacles(P):
    """Trunks spanning the workspace along one axis give a broad-phase grid
    flat along that axis; walls of small tiles keep the cube.  With the
    forest turned so that its trunks run along x or along y, lock-step
    passes still match the oracle's test of every box."""
    assert P.Planner(W.c2(0)).info()["bp_grid"] == [64, 64, 1]
    assert P.Planner(W.c3(0)).info()["bp_grid"] == [16, 16, 16]
    trunks = W.c2(0).boxes
    for order, want in (((2, 0, 1), [1, 64, 64]), ((0, 2, 1), [64, 1, 64])):
        boxes = np.concatenate([trunks[:, list(order)], trunks[:, [3 + a for a in order]]], 1)
        w = W.tiny(W.DI, seed=0, t_e=4000, lambda_max=16, n_boxes=0)
        p0 = w.x_init[:3]
        keep = ~np.all((boxes[:, :3] <= p0 + 0.06) & (boxes[:, 3:] >= p0 - 0.06), axis=1)
        w = w.with_(boxes=np.ascontiguousarray(boxes[keep]))
        assert P.Planner(w).info()["bp_grid"] == want
        exact, ran, flips, n, _ = lockstep(P, w, 6)
        assert exact >= min(ran, 2)


def test_boxes_on_cell_faces(P):
    """Boxes whose faces sit exactly on broad-phase cell faces (multiples
    of 1/16) and a sample path along them: verdicts match the oracle."""
    boxes = []
    for i in range(1, 15, 3):
        for j in range(1, 15, 4):
            boxes.append([i / 16, j / 16, 0.0, (i + 1) / 16, (j + 1) / 16, 1.0])
    boxes = np.asarray(boxes, np.float32)
    w = W.tiny(W.DI, seed=0, t_e=4000, lambda_max=16, n_boxes=0).with_(
        boxes=boxes, x_init=np.array([0.03, 0.03, 0.5, 0, 0, 0], np.float32))
    exact, ran, flips, n, _ = lockstep(P, w, 8)
    assert exact >= min(ran, 3)


def test_grow_keeps_tree_and_continues_in_lockstep(P):
    """Remark 1 (adaptive node cap): the oracle fills a tree at t_e = 2048
    (Eq. 6 gives lambda = 0); the device context holding it moves to a 4x
    cap.  The tree, tables and loop state survive the move unchanged, and
    the next pass matches the oracle continuing its own tree with the new
    cap."""
    w = W.c1(1, t_e=2048)
    src = Oracle(w)
    src.reset()
    for _ in range(60):
        status, _, _ = src.iterate()
        if status != kpo.RUNNING:
            break
    assert status == kpo.FULL
    t = src.export()
    t["state"] = t["state"].astype(np.float32)
    t["ctrl"] = t["ctrl"].astype(np.float32)
    g = P.Planner(w)
    g.import_tree(t)
    st, _ = g.resume(max_iters=5)
    assert st == P.NO_SOLUTION and g.info()["state"] == 2  # still full
    g.grow(4 * w.t_e)
    after = g.export_tree()
    for key in ("parent", "steps", "region", "sub", "in_ve", "n_valid", "n_invalid", "thr",
                "visited", "cov", "avail"):
        assert np.array_equal(after[key], t[key]), key
    assert np.array_equal(after["state"], t["state"]) and np.array_equal(after["ctrl"], t["ctrl"])
    w2 = w.with_(t_e=4 * w.t_e)
    o = Oracle(w2)
    o.import_(t)
    g.enable_log(w2.t_e)
    status, ost, orec = o.iterate(records=True)
    gs = g.expand_step(1)
    assert len(gs) == 1 and ost["n_samples"] > 0
    assert compare_pass(w2, ost, orec, gs[0], g.read_log(ost["n_samples"])) <= 2


@pytest.mark.parametrize("seed", [0, 2])
def test_plan_adaptive_revalidated(P, seed):
    """A cap too small for the double-integrator query grows by 2x until a
    goal node is reached; the trajectory re-validates under the oracle."""
    w = W.c1(seed, t_e=2048)
    g = P.Planner(w)
    st, traj, grown = g.plan_adaptive(max_iters=400, growth=2.0, t_e_max=1 << 18)
    assert st == P.OK and grown >= 1
    o = Oracle(w)
    scale = state_scale(w)
    prev = w.x_init.astype(np.float64)
    for e in range(len(traj["steps"])):
        depth, x_end = o.dense_check(prev, traj["ctrls"][e].astype(np.float64),
                                     int(traj["steps"][e]), 100)
        assert depth <= 1e-4
        assert np.max(np.abs(x_end - traj["states"][e]) / scale) <= 1e-4
        prev = traj["states"][e].astype(np.float64)
    assert np.linalg.norm(prev[:3] - w.goal_c) <= float(w.goal_r) * (1 + 1e-6)


def _state_grid(**cells):
    sg = [0] * 12
    for d, n in cells.items():
        sg[int(d[1:])] = n
    return tuple(sg)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lockstep_tiny_state_grid(P, seed):
    """Regions over the whole Dubins state (Sec. VI): 2^3 position cells x
    4 heading cells (wrapped angle) x 2 pitch x 2 speed cells."""
    w = W.tiny(W.DUBINS, seed=seed, t_e=2000, lambda_max=8,
               state_grid=_state_grid(d3=4, d4=2, d5=2))
    exact, ran, flips, n, _ = lockstep(P, w, 12)
    assert exact >= min(ran, 3)


def test_frontier_c2_state_grid(P):
    """The Dubins forest with an 8^3 x 4 x 2 x 2 state-space grid (8,192
    regions, 524,288 sub-regions): one pass over the oracle's 3-pass tree."""
    w = W.c2(0, grid=(8, 8, 8), state_grid=_state_grid(d3=4, d4=2, d5=2))
    flips, ost = frontier(P, w, grow=2)
    assert ost["n_samples"] > 10000
    assert flips <= 2


# ---------------------------------------------------------------------------
# free-space-obeying decomposition (kd-tree over obstacle faces, Sec. IV-B)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("system", [W.DI, W.DUBINS, W.QUAD])
@pytest.mark.parametrize("seed", [0, 1])
def test_lockstep_tiny_fso(P, system, seed):
    """Regions are the leaves of the kd-tree the host builds from the
    obstacles; each pass matches the oracle's own tree and leaf volumes."""
    w = W.tiny(system, seed=seed, t_e=2000, lambda_max=8, n_boxes=4, fso=True)
    g = P.Planner(w)
    assert g.n_regions == Oracle(w).R > 1
    exact, ran, flips, n, _ = lockstep(P, w, 12)
    assert exact >= min(ran, 3)


def test_lockstep_c1_fso(P):
    """Double integrator, 16 random boxes: kd-tree regions, passes of up to
    tens of thousands of samples."""
    w = W.c1(1).with_(fso=True)
    exact, ran, flips, n, _ = lockstep(P, w, 10)
    assert exact >= ran // 2, (exact, ran, flips, n)
    assert flips <= 1e-4 * n


def test_frontier_c2_fso(P):
    """The 200-trunk Dubins forest with kd-tree regions (about 1,240
    leaves): one pass over the oracle's 3-pass tree."""
    w = W.c2(0).with_(fso=True)
    flips, ost = frontier(P, w, grow=2)
    assert ost["n_samples"] > 10000
    assert flips <= 2


def test_frontier_c3_fso(P):
    """The 1,200-box quadrotor building with kd-tree regions (about 2,000
    leaves): one pass over the oracle's 1-pass tree."""
    w = W.c3(0).with_(fso=True)
    flips, ost = frontier(P, w, grow=1)
    assert ost["n_samples"] > 10000
    assert flips <= 2


def test_fso_obstacle_swap_rebuilds(P):
    """kp_set_obstacles rebuilds the tree: the region count follows the new
    set (as the oracle builds it), planning re-validates, and an empty set
    is one region (the whole workspace: no guidance, so a short budget need
    not solve)."""
    w = W.c1(0).with_(fso=True)
    empty = w.with_(boxes=np.zeros((0, 6), np.float32))
    g = P.Planner(empty, box_capacity=64)
    assert g.n_regions == 1
    st, _ = g.plan(max_iters=20)
    assert st in (P.OK, P.NO_SOLUTION)
    _tree_invariants(empty, g.export_tree())
    g.set_obstacles(w.boxes)
    g.w = w
    assert g.n_regions == Oracle(w).R
    st, traj = g.plan(max_iters=200)
    assert st == P.OK
    _revalidate(w, traj, w.x_init)
    _tree_invariants(w, g.export_tree(), sample_edges=200)


@pytest.mark.parametrize("seed", [0, 1])
def test_plan_c2_fso_revalidated(P, seed):
    """Full-size forest query with kd-tree regions: trajectory re-validated
    by the oracle, and the tree's regions are the oracle's leaves."""
    w = W.c2(seed).with_(fso=True)
    g = P.Planner(w)
    st, traj = g.plan(max_iters=200)
    assert st == P.OK
    _revalidate(w, traj, w.x_init)
    _tree_invariants(w, g.export_tree(), sample_edges=300, info=g.info())


def test_grow_fso_keeps_leaves(P):
    """Remark 1 with kd-tree regions: after the move to a larger arena the
    next pass still bins into the same leaves as the oracle."""
    w = W.c1(1, t_e=1024).with_(fso=True)
    src = Oracle(w)
    src.reset()
    for _ in range(60):
        status, _, _ = src.iterate()
        if status != kpo.RUNNING:
            break
    assert status == kpo.FULL
    t = src.export()
    t["state"] = t["state"].astype(np.float32)
    t["ctrl"] = t["ctrl"].astype(np.float32)
    g = P.Planner(w)
    g.import_tree(t)
    g.grow(4 * w.t_e)
    w2 = w.with_(t_e=4 * w.t_e)
    o = Oracle(w2)
    o.import_(t)
    g.enable_log(w2.t_e)
    status, ost, orec = o.iterate(records=True)
    gs = g.expand_step(1)
    assert len(gs) == 1 and ost["n_samples"] > 0
    assert compare_pass(w2, ost, orec, gs[0], g.read_log(ost["n_samples"])) <= 2
    compare_trees(w2, g.export_tree(), o.export())



# ---------------------------------------------------------------------------
# whole queries, statistically: device vs oracle over 100 seeds
# ---------------------------------------------------------------------------

def _oracle_full_run(seed):
    """(solved, passes, |T|) of the oracle's whole C1 query (run in a spawned
    worker: module-level so that it pickles by name)."""
    o = Oracle(W.c1(seed))
    o.reset()
    status, passes = o.run(200)
    return status == kpo.SOLVED, passes, o.n_nodes


def _ks(a, b):
    """Two-sample Kolmogorov-Smirnov statistic."""
    a, b = np.sort(np.asarray(a, float)), np.sort(np.asarray(b, float))
    grid = np.concatenate([a, b])
    fa = np.searchsorted(a, grid, side="right") / len(a)
    fb = np.searchsorted(b, grid, side="right") / len(b)
    return float(np.max(np.abs(fa - fb)))


def test_whole_queries_match_oracle_statistically(P):
    """Whole queries cannot match exactly (FP32 against FP64 decisions near
    a face eventually split the trees), so C1 queries on 100 seeds are
    compared in law: success rate, passes to solve and tree size at the
    solution.  The two-sample KS statistic must stay below its 0.1 %
    critical value (1.95 sqrt(2/100) = 0.276), and most seeds must run the
    same number of passes (lock-step passes match exactly until a split)."""
    import multiprocessing as mp
    import os
    seeds = list(range(100, 200))
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        orc = pool.map(_oracle_full_run, seeds, chunksize=1)
    dev = []
    for s in seeds:
        w = W.c1(s)
        g = P.Planner(w)
        st, _ = g.plan(max_iters=200)
        info = g.info()
        dev.append((st == P.OK, info["iteration"], info["n_nodes"]))
        g.close()
    o_ok = np.array([r[0] for r in orc])
    d_ok = np.array([r[0] for r in dev])
    assert abs(o_ok.mean() - d_ok.mean()) <= 0.05
    o_it, d_it = [r[1] for r in orc], [r[1] for r in dev]
    o_n, d_n = [r[2] for r in orc], [r[2] for r in dev]
    assert _ks(o_it, d_it) <= 0.276, (_ks(o_it, d_it), np.mean(o_it), np.mean(d_it))
    assert _ks(o_n, d_n) <= 0.276, (_ks(o_n, d_n), np.mean(o_n), np.mean(d_n))
    assert abs(np.mean(o_n) / np.mean(d_n) - 1.0) <= 0.1
    same = np.mean(np.array(o_it) == np.array(d_it))
    assert same >= 0.5, same


def test_fso_leaf_capacity_refused_and_context_unchanged(P):
    """An obstacle set whose kd-tree passes 16,384 leaves is refused with
    KP_ERR_ARG, at creation and on replacement; a refused replacement
    leaves the context as it was (same regions, plans as before)."""
    rng_boxes = lambda n: W.random_boxes(5, n, side=(0.01, 0.03),
                                         keep_clear=[((0.1, 0.1, 0.1), 0.02),
                                                     ((0.9, 0.9, 0.9), 0.06)])
    w = W.c1(0).with_(fso=True)
    with pytest.raises(P.KpError) as e:
        P.Planner(w.with_(boxes=rng_boxes(2000)))
    assert e.value.status == P.ERR_ARG
    g = P.Planner(w, box_capacity=2000)
    regions = g.n_regions
    assert regions == Oracle(w).R
    with pytest.raises(P.KpError) as e:
        g.set_obstacles(rng_boxes(2000))
    assert e.value.status == P.ERR_ARG
    assert g.info()["n_regions"] == regions
    st, traj = g.plan(max_iters=200)
    assert st == P.OK
    _revalidate(w, traj, w.x_init)
    _tree_invariants(w, g.export_tree(), sample_edges=100)


def test_measured_lane_peak_near_the_derived_one(P):
    """The FMA microbenchmark (the measured ALU denominator) lands near SMs x
    128 lanes x the maximum SM clock (2,070 MHz on this part): above 40 %
    of it (clocks may sit below the maximum) and not above it by more than
    the timing noise."""
    import torch
    v = P.measure_lane_peak()
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    derived = n_sm * 128 * 2070e6
    assert 0.4 * derived <= v <= 1.05 * derived, (v, derived)
