"""The oracle's work counts (oracle/work.c) against the oracle's own replay
records and against cases whose counts are known: the algorithmic work the
benchmark's roofline reports is the oracle's count, so the count itself is
pinned here."""
import numpy as np
import pytest

from oracle.kpo import Oracle
from paper_2409_06807_gb300 import workloads as W


@pytest.mark.parametrize("system", [W.DI, W.DUBINS, W.QUAD])
def test_oracle_work_counts_agree_with_its_replay_records(system):
    """The oracle's work counters (oracle/work.c, fed by hooks in the
    replay) against the per-sample records of the same replay: one sample
    counted per drawn sample, the steps a sample ran (its duration, or the
    step at which it failed), and one hull per step except a failing step
    whose end state left the state box.  A pass with an empty obstacle set
    tests no box; with a single box the plain scan tests exactly one box
    per hull."""
    w = W.tiny(system, seed=4)
    o = Oracle(w)
    o.set_work_grid((16, 16, 16))
    o.reset()
    n = steps = hulls = 0
    lo, hi = w.x_lo[: o.d].astype(np.float64), w.x_hi[: o.d].astype(np.float64)
    for _ in range(3):
        _, st, rec = o.iterate(records=True)
        n += st["n_samples"]
        fail, k = rec["fail_step"], rec["k"]
        run = np.where(fail > 0, fail, k)
        steps += int(run.sum())
        out = np.any((rec["state"] < lo) | (rec["state"] > hi), axis=1) & (fail > 0)
        hulls += int(run.sum() - out.sum())
    wk = o.work()
    assert wk["samples"] == n > 0
    assert wk["steps"] == steps
    assert wk["hulls"] == hulls
    # no obstacles: nothing to test
    e = Oracle(w.with_(boxes=np.zeros((0, 6), np.float32)))
    e.set_work_grid((16, 16, 16))
    e.reset()
    e.iterate()
    assert e.work()["box_scan"] == 0 and e.work()["box_grid"] == 0
    assert e.work()["hulls"] > 0
    # one box: the plain scan tests it once per hull, met or not
    one = W.tiny(system, seed=4, n_boxes=1)
    b = Oracle(one)
    b.set_work_grid((16, 16, 16))
    b.reset()
    for _ in range(2):
        b.iterate()
    assert b.work()["box_scan"] == b.work()["hulls"] > 0
