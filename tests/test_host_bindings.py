"""Host-side logic of the Python binding that needs no GPU: the network's
parameter layout (shared by the C ABI and the oracle, each counting it on
its own) and the serving summary's statistics."""
import numpy as np
import pytest

from oracle import kpo
from paper_2409_06807_gb300 import mlp, serve
from paper_2409_06807_gb300.planner import NO_SOLUTION, OK


@pytest.fixture(scope="module", autouse=True)
def built():
    """The planner library (cross-compiled for sm_103a; only host entry
    points are called here)."""
    from paper_2409_06807_gb300.build import build_planner
    return build_planner()


def test_network_parameter_layout_matches_the_oracle():
    p = mlp.init_params(0)
    assert p.size == mlp.num_params() == kpo.mlp_num_params()
    ours = [b.shape for b in mlp.split(p)]
    theirs = [b.shape for b in kpo.mlp_split(p.astype(np.float64))]
    assert ours == theirs
    # He-uniform hidden layers, a 0.1-gain output layer, zero biases
    W1, b1, W2, b2, W3, b3 = mlp.split(p)
    assert np.abs(W1).max() <= np.sqrt(6.0 / W1.shape[1]) and np.abs(W3).max() <= 0.1 * np.sqrt(6.0 / W3.shape[1])
    assert not b1.any() and not b2.any() and not b3.any()
    assert np.array_equal(mlp.init_params(0), p) and not np.array_equal(mlp.init_params(1), p)


def test_serving_summary():
    lat = np.arange(1, 101, dtype=np.float64)  # 1 .. 100 ms
    recs = [dict(latency_ms=float(x), status=OK if i % 4 else NO_SOLUTION, samples=1000)
            for i, x in enumerate(lat)]
    s = serve.summarize(recs, wall_s=0.5)
    assert s["queries"] == 100 and s["success"] == pytest.approx(0.75)
    assert s["p50_ms"] == pytest.approx(np.percentile(lat, 50))
    assert s["p99_ms"] == pytest.approx(np.percentile(lat, 99))
    assert s["queries_per_s"] == pytest.approx(200.0) and s["samples_per_s"] == pytest.approx(2e5)
    assert s["status"] == {"OK": 75, "NO_SOLUTION": 25}
