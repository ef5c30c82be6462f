"""Batched planning in one persistent launch (teams of blocks), continuous
admission, and result independence from co-running queries."""
import numpy as np
import pytest

from oracle.kpo import Oracle
from paper_2409_06807_gb300 import workloads as W
from parity_util import state_scale

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2409_06807_gb300.build import build_planner
    build_planner()
    from paper_2409_06807_gb300 import planner, serve
    return planner, serve


def _mix():
    qs = []
    for s in range(4):
        qs.append(W.c1(s))
        qs.append(W.c2(s, t_e=1 << 18))
        qs.append(W.c3(s, t_e=1 << 17, lambda_max=32))
    return qs


def _same(a, b):
    return (len(a["steps"]) == len(b["steps"]) and np.array_equal(a["steps"], b["steps"])
            and np.array_equal(a["states"], b["states"]) and np.array_equal(a["ctrls"], b["ctrls"]))


def test_alone_and_in_the_mix_are_identical(S):
    """Twelve queries of the three systems run together; each is then run
    alone through the same server: identical status and trajectory."""
    P, serve = S
    qs = _mix()
    srv = serve.Server(4 << 30, team_blocks=16, max_slots=64, idle_ms=50)
    ids = [srv.submit(w, max_iters=60) for w in qs]
    done = {d["id"]: d for d in srv.drain()}
    mixed = {i: srv.result(i) for i in ids}
    assert all(done[i]["status"] in (P.OK, P.NO_SOLUTION) for i in ids)
    assert sum(done[i]["status"] == P.OK for i in ids) >= 6
    for w, i in zip(qs, ids):
        j = srv.submit(w, max_iters=60)
        d = srv.drain()
        assert len(d) == 1 and d[0]["status"] == done[i]["status"]
        assert d[0]["samples"] == done[i]["samples"]
        alone = srv.result(j)
        assert alone[0] == mixed[i][0]
        assert _same(alone[1], mixed[i][1])
    srv.close()


def test_server_results_revalidated_and_match_single_launch(S):
    """Solved server queries re-validate under the oracle; the single-query
    launch on the same inputs returns the same trajectory bit for bit.  Both
    run the same explicitly rounded FP32 arithmetic on the same keys, and
    the obstacle test's verdict is exact whatever the broad-phase grid (the
    server's blob is built without cell clearances, within its 48 KB room),
    so status, edge count, states, controls and durations must agree
    exactly."""
    P, serve = S
    qs = [W.c1(s) for s in range(3)] + [W.c2(s, t_e=1 << 18) for s in range(2)]
    srv = serve.Server(4 << 30, team_blocks=32, max_slots=16, idle_ms=50)
    ids = [srv.submit(w, max_iters=100) for w in qs]
    srv.drain()
    for w, i in zip(qs, ids):
        st, tr = srv.result(i)
        st1, tr1 = P.Planner(w).plan(max_iters=100)
        assert st1 == st
        if st != P.OK:
            continue
        o = Oracle(w)
        scale = state_scale(w)
        prev = w.x_init.astype(np.float64)
        for e in range(len(tr["steps"])):
            depth, x_end = o.dense_check(prev, tr["ctrls"][e].astype(np.float64),
                                         int(tr["steps"][e]), 100)
            assert depth <= 1e-4
            assert np.max(np.abs(x_end - tr["states"][e]) / scale) <= 1e-4
            prev = tr["states"][e].astype(np.float64)
        assert np.linalg.norm(prev[:3] - w.goal_c) <= float(w.goal_r) * (1 + 1e-6)
        assert _same(tr1, tr), (len(tr1["steps"]), len(tr["steps"]))
    srv.close()


def test_admission_waits_for_pool_memory(S):
    """A pool that holds only a few query arenas at once: the rest wait in
    submission order and are admitted as memory frees; all complete."""
    P, serve = S
    w = W.c1(0)
    per = P.lib().kp_required_bytes(*[__import__("ctypes").byref(x) for x in P.structs(w)[:2]],
                                    len(w.boxes), __import__("ctypes").byref(P.structs(w)[2]))
    ctl = P.lib().kp_server_required_bytes(16)
    srv = serve.Server(ctl + 3 * per + (1 << 20), team_blocks=16, max_slots=16, idle_ms=50)
    ids = [srv.submit(W.c1(s), max_iters=100) for s in range(10)]
    assert srv.stats()["pending"] >= 6
    done = srv.drain()
    assert sorted(d["id"] for d in done) == sorted(ids)
    assert all(d["status"] in (P.OK, P.NO_SOLUTION) for d in done)
    srv.close()


def test_invalid_queries_complete_with_errors(S):
    P, serve = S
    srv = serve.Server(1 << 30, team_blocks=16, max_slots=8, idle_ms=50)
    w = W.c1(0)
    bad = w.x_init.copy()
    bad[3] = 9.0  # velocity outside its bound
    i_bad = srv.submit(w.with_(x_init=bad))
    i_ok = srv.submit(w)
    done = {d["id"]: d for d in srv.drain()}
    assert done[i_bad]["status"] == P.ERR_ARG
    assert done[i_ok]["status"] == P.OK
    srv.close()


def test_serving_run_reports_latency(S):
    """A short Poisson arrival run (continuous batching): every query
    completes and latencies are recorded."""
    P, serve = S
    import time
    arrivals = W.serving_mix(48, rate_hz=2000.0, seed=3, t_e_range=(16384, 1 << 18),
                             box_range=(10, 300))
    srv = serve.Server(8 << 30, team_blocks=16, max_slots=64, idle_ms=100)
    t0 = time.perf_counter()
    recs = serve.run_arrivals(srv, arrivals, max_iters=60)
    summ = serve.summarize(recs, time.perf_counter() - t0)
    assert summ["queries"] == 48 and summ["p99_ms"] >= summ["p50_ms"] > 0
    srv.close()
