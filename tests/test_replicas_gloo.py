"""The multi-rank path on CPU (gloo, world size 2): each rank plans its own
seeded layouts (replicas, no data-path exchange); the whole-job rate is
the units of all ranks over the slowest rank's time; under torchrun only
rank 0 prints the one JSON line."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units = [1000.0, 3000.0][rank]
    ms = [40.0, 100.0][rank]
    out = {
        "max": bench.max_over_ranks(ms, world),
        "sum": bench.sum_over_ranks(units, world),
        "rate": bench.whole_job_rate(units, ms, world),
        "seeds": bench.rank_seeds(rank, 5),
    }
    bench.barrier(world)
    dist.destroy_process_group()
    q.put((rank, out))


def test_rank_reductions_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        assert res[r]["max"] == 100.0
        assert res[r]["sum"] == 4000.0
        assert res[r]["rate"] == pytest.approx(4000.0 / 0.1)
    assert not set(res[0]["seeds"]) & set(res[1]["seeds"])
    assert res[0]["seeds"] == list(range(5))


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.sum_over_ranks(3.0, 1) == 3.0
    assert bench.whole_job_rate(500.0, 250.0, 1) == pytest.approx(2000.0)


def test_reference_arm_under_torchrun_prints_once():
    """Two ranks launched as the benchmark harness launches them: rank 0
    times the CPU oracle and prints one line, rank 1 exits cleanly."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--gpus", "2",
           "--impl", "reference", "--workload", "c1", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
