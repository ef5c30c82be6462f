"""Host logic of the benchmark: the algorithmic work per unit behind the
roofline, the clock record's throttle detection, the measured-peak lookup
and the rule that a stored DRAM traffic figure is used only for the kernel
sources it was taken on."""
import os

import pytest

import bench
from oracle.kpo import Oracle
from paper_2409_06807_gb300 import workloads as W


def test_algorithmic_work_per_unit():
    # per sample, per integrator step, per step hull, per hull-vs-box test
    for system, sample, step in ((W.DI, 157, 18), (W.DUBINS, 157, 127), (W.QUAD, 173, 337)):
        assert bench.alg_ops(system, 1, 0, 0, 0) == sample
        assert bench.alg_ops(system, 0, 1, 0, 0) == step
        assert bench.alg_ops(system, 0, 0, 1, 0) == 6
        assert bench.alg_ops(system, 0, 0, 0, 1) == 8
    # linear in every count
    assert bench.alg_ops(W.DUBINS, 10, 63, 63, 95) == 10 * 157 + 63 * 127 + 63 * 6 + 95 * 8


@pytest.mark.parametrize("make,passes,grid", [(W.c1, 4, (16, 16, 16)), (W.c2, 3, (64, 64, 1)),
                                              (W.c3, 2, (16, 16, 16))])
def test_algorithmic_work_equals_the_oracle_replay_count(make, passes, grid):
    """The roofline's work per unit is the oracle's: the oracle counts
    samples, integrator steps, step hulls and broad-phase box tests as it
    replays seeded passes (oracle/work.c), and costs each under the same
    counting rule; the benchmark's table applied to those counts gives the
    oracle's total exactly."""
    w = make(3)
    o = Oracle(w)
    o.set_work_grid(grid)
    o.reset()
    for _ in range(passes):
        o.iterate()
    wk = o.work()
    assert wk["samples"] > 0 and wk["steps"] >= wk["hulls"] > 0 and wk["box_grid"] > 0
    assert o.work_costs() == {"sample": bench.OPS_PER_SAMPLE[w.system],
                              "step": bench.OPS_PER_STEP[w.system],
                              "hull": bench.OPS_PER_HULL, "box": bench.OPS_PER_BOX}
    assert bench.alg_ops(w.system, wk["samples"], wk["steps"], wk["hulls"],
                         wk["box_grid"]) == wk["ops"]
    # the broad phase tests far fewer boxes than a scan of every box
    assert wk["box_grid"] < wk["box_scan"]


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.lines = lines
    return s.summary()


def test_clock_summary_flags_throttle_reasons():
    ok = "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active"
    hot = "0, 1500, 2070, 1390.0, 0x40, Not Active, Active, Not Active, Not Active"
    s = _sampler([ok, ok, ok])
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070 and s["reasons"] == []
    s = _sampler([ok, capped, capped])
    assert s["sm_mhz"] == 1980 and s["reasons"] == ["sw_power_cap"]
    s = _sampler([ok, hot, "garbage", "0, [N/A], 2070, 1, 0, a, b, c, d"])
    assert s["reasons"] == ["hw_thermal_slowdown"] and s["samples"] == 2
    assert _sampler([])["reasons"] == ["unsampled"]


def _tree(tmp_path, src=b"kernel v1"):
    csrc = tmp_path / "paper_2409_06807_gb300" / "csrc"
    csrc.mkdir(parents=True, exist_ok=True)
    (csrc / "k.cu").write_bytes(src)
    (tmp_path / "profiles").mkdir(exist_ok=True)
    return csrc


def test_traffic_only_for_the_sources_it_was_taken_on(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    csrc = _tree(tmp_path)
    h = bench.source_hash()
    (tmp_path / "profiles" / "k.traffic").write_text(
        f"# dram bytes of one launch\nsource_hash: {h}\ndram_bytes_per_launch: 1234.5\n")
    assert bench.profiled_traffic("k") == 1234.5
    assert bench.profiled_traffic("missing") is None
    (csrc / "k.cu").write_bytes(b"kernel v2")
    assert bench.source_hash() != h
    assert bench.profiled_traffic("k") is None


def test_peaks_fall_back_when_unmeasured(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    p, kind = bench.peaks()
    assert kind == "fallback" and p["hbm_gbs"] == 6800.0 and p["bf16_tflops"] == 1900.0
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 7000.0}')
    p, kind = bench.peaks()
    assert kind == "measured" and p["hbm_gbs"] == 7000.0


def test_committed_traffic_records_name_a_source_hash():
    prof = os.path.join(os.path.dirname(bench.__file__), "profiles")
    files = [f for f in os.listdir(prof) if f.endswith(".traffic")]
    assert files
    for f in files:
        with open(os.path.join(prof, f)) as fh:
            keys = {ln.split(":", 1)[0].strip() for ln in fh if ":" in ln and not ln.startswith("#")}
        assert {"source_hash", "dram_bytes_per_launch"} <= keys, f

