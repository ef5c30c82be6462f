"""kp_plan_static: the planning query for callers that cannot allocate.

Some callers may not allocate device memory at all (a host application
that owns all device memory through its own pool, a plugin inside such a
process, a real-time control loop that cannot afford an allocation's
implicit synchronisation).  kp_plan_static serves them from a fixed static
device scratch.  These tests call it through the C ABI and check that it
returns what the arena-based kp_plan returns for the same query, on two
calls in a row (the second call runs on the scratch the first one left
behind), and that an oversized problem is refused before any device work.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2409_06807_gb300 import workloads as W
from parity_util import state_scale

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2409_06807_gb300.build import build_planner
    build_planner()
    from paper_2409_06807_gb300 import planner
    return planner


def static_plan(P, w, max_iters=200, capacity=1024):
    import torch
    sys_, ws, prm = P.structs(w)
    boxes = np.ascontiguousarray(np.asarray(w.boxes, np.float32).reshape(-1, 6))
    obs = P.Obstacles(boxes.ctypes.data_as(C.POINTER(C.c_float)) if len(boxes) else None,
                      len(boxes))
    x = np.ascontiguousarray(w.x_init, np.float32)
    g = P.goal_struct(w)
    b = P.Budget(max_iters, 0.0)
    states = np.zeros((capacity, 12), np.float32)
    ctrls = np.zeros((capacity, 4), np.float32)
    steps = np.zeros(capacity, np.int32)
    t = P.Traj(capacity, 0, states.ctypes.data_as(C.POINTER(C.c_float)),
               ctrls.ctypes.data_as(C.POINTER(C.c_float)),
               steps.ctypes.data_as(C.POINTER(C.c_int32)))
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = P.lib().kp_plan_static(C.byref(sys_), C.byref(ws), C.byref(obs), C.byref(prm),
                                x.ctypes.data_as(C.POINTER(C.c_float)), C.byref(g), C.byref(b),
                                C.byref(t), stream)
    n = t.n_edges
    return st, dict(states=states[:n, : w.d], ctrls=ctrls[:n, : w.n_ctrl], steps=steps[:n])


def _same_as_kp_plan(P, w, max_iters=200):
    st_ref, ref = P.Planner(w).plan(max_iters=max_iters, capacity=1024)
    st, got = static_plan(P, w, max_iters=max_iters)
    assert st == st_ref
    assert np.array_equal(got["steps"], ref["steps"])
    scale = state_scale(w)
    if len(got["steps"]):
        assert np.max(np.abs(got["states"] - ref["states"]) / scale) <= 1e-4
        span = np.asarray(w.u_hi[: w.n_ctrl]) - np.asarray(w.u_lo[: w.n_ctrl])
        assert np.max(np.abs(got["ctrls"] - ref["ctrls"]) / span) <= 1e-6
    return st, got


def _revalidate(w, traj):
    """Every returned edge re-propagated in FP64 from its parent state by the
    oracle and checked densely (100 sub-steps per integrator step)."""
    from oracle.kpo import Oracle
    o = Oracle(w)
    scale = state_scale(w)
    prev = np.asarray(w.x_init, np.float64)
    for e in range(len(traj["steps"])):
        depth, x_end = o.dense_check(prev, traj["ctrls"][e].astype(np.float64),
                                     int(traj["steps"][e]), 100)
        assert depth <= 1e-4, f"edge {e} penetrates by {depth}"
        assert np.max(np.abs(x_end - traj["states"][e]) / scale) <= 1e-4
        prev = traj["states"][e].astype(np.float64)
    assert np.linalg.norm(prev[:3] - w.goal_c) <= float(w.goal_r) * (1 + 1e-6)


def test_static_plan_matches_kp_plan_on_consecutive_calls(P):
    for seed in (0, 1):  # two calls in a row share the static scratch
        st, got = _same_as_kp_plan(P, W.c1(seed))
        assert st == P.OK
        _revalidate(W.c1(seed), got)


def test_static_plan_calls_of_changing_shape(P):
    """Calls whose shapes differ share the scratch: a Dubins forest query
    (4,096 regions, 200 boxes), a double-integrator query (512 regions, 16
    boxes), the forest again, and a forest query over an 8,192-region state
    grid.  The scratch keeps what the larger call left (tables, box rows,
    the grid); each call must still return kp_plan's result, and every
    solved trajectory re-validates under the oracle."""
    sg = (0, 0, 0, 4, 2, 2, 0, 0, 0, 0, 0, 0)
    seq = [W.c2(3, t_e=60000, lambda_max=32), W.c1(1), W.c2(3, t_e=60000, lambda_max=32),
           W.c2(5, t_e=40000, lambda_max=32, grid=(8, 8, 8), state_grid=sg)]
    solved = 0
    for w in seq:
        st, got = _same_as_kp_plan(P, w)
        if st == P.OK:
            solved += 1
            _revalidate(w, got)
    assert solved >= 3


def test_static_plan_refuses_oversized_problem(P):
    w = W.c2(0)  # t_e = 2^20: its arena is far above the static maximum
    st, _ = static_plan(P, w)
    assert st == P.ERR_OOM


def test_static_plan_takes_grid_regions_only(P):
    """The kd-tree decomposition needs the context path (its tree is built
    with the obstacles); the no-allocation entry point refuses it."""
    st, _ = static_plan(P, W.c1(0).with_(fso=True))
    assert st == P.ERR_ARG
