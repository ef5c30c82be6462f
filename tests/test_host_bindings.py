"""Host-side logic that needs no GPU: the network's parameter layout
(shared by the C ABI and the oracle, each counting it on its own), the
serving summary's statistics, the C ABI's argument validation and the
arena's size per tree node."""
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


def test_serving_summary_by_system():
    """Failures are attributed to their system with the node caps they had."""
    recs = []
    for i in range(30):
        sysid = i % 3
        t_e = 1 << (14 + i % 7)
        ok = not (sysid == 2 and t_e < (1 << 19))
        recs.append(dict(latency_ms=float(i + 1), status=OK if ok else NO_SOLUTION,
                         samples=10, system=sysid, t_e=t_e, boxes=10))
    by = serve.summarize_by_system(recs)
    assert sorted(by) == ["0", "1", "2"]
    assert by["0"]["success"] == 1.0 and by["0"]["failures"] == 0
    assert by["0"]["failed_t_e_median"] is None
    fails = [r for r in recs if r["system"] == 2 and r["status"] != OK]
    assert by["2"]["failures"] == len(fails) > 0
    assert by["2"]["failed_t_e_median"] == float(np.median([r["t_e"] for r in fails]))
    assert by["2"]["queries"] == 10 and by["2"]["success"] == (10 - len(fails)) / 10


def _required(w, n_boxes=None, edit=None):
    import ctypes as C
    from paper_2409_06807_gb300 import planner
    s, ws, p = planner.structs(w)
    if edit:
        edit(s, ws, p)
    return planner.lib().kp_required_bytes(C.byref(s), C.byref(ws),
                                           len(w.boxes) if n_boxes is None else n_boxes,
                                           C.byref(p))


def _set(obj, field, value, index=None):
    if index is None:
        setattr(obj, field, value)
    else:
        getattr(obj, field)[index] = value


NAN = float("nan")
INVALID = {
    "dt zero": ("s", "dt", 0.0, None), "dt NaN": ("s", "dt", NAN, None),
    "k_min zero": ("s", "k_min", 0, None), "k_max below k_min": ("s", "k_max", 0, None),
    "k_max above 255": ("s", "k_max", 256, None),
    "state bound NaN": ("s", "x_lo", NAN, 4), "state bounds crossed": ("s", "x_lo", 1.0, 4),
    "control bounds crossed": ("s", "u_lo", 2.0, 0), "control bound infinite": ("s", "u_hi", float("inf"), 1),
    "workspace empty": ("ws", "hi", 0.0, 0), "grid zero": ("ws", "grid", 0, 1),
    "grid above 4096": ("ws", "grid", 4097, 2), "sub zero": ("ws", "sub", 0, 0),
    "speed bins zero": ("ws", "speed_bins", 0, None), "fso two": ("ws", "fso", 2, None),
    "state grid negative": ("ws", "state_grid", -1, 4),
    "t_e one": ("p", "t_e", 1, None), "t_e above 2^28": ("p", "t_e", (1 << 28) + 1, None),
    "lambda zero": ("p", "lambda_max", 0, None), "lambda above 1024": ("p", "lambda_max", 1025, None),
    "delta zero": ("p", "delta", 0.0, None), "eps zero": ("p", "eps", 0.0, None),
    "eps one": ("p", "eps", 1.0, None),
}


@pytest.mark.parametrize("case", sorted(INVALID))
def test_inputs_are_validated_on_the_host(case):
    """Every documented argument error makes kp_required_bytes return 0 (the
    same check kp_create applies before touching the device)."""
    from paper_2409_06807_gb300 import workloads as W
    which, field, value, index = INVALID[case]
    w = W.c2(0)
    assert _required(w) > 0

    def edit(s, ws, p):
        _set({"s": s, "ws": ws, "p": p}[which], field, value, index)
    assert _required(w, edit=edit) == 0


def test_box_count_and_decomposition_limits():
    from paper_2409_06807_gb300 import planner
    from paper_2409_06807_gb300 import workloads as W
    w = W.c2(0)
    assert _required(w, n_boxes=-1) == 0
    assert _required(w, n_boxes=planner.MAX_BOXES) > 0 and _required(w, n_boxes=planner.MAX_BOXES + 1) == 0

    def speed_without_range(s, ws, p):
        ws.speed_bins, ws.speed_hi = 4, 0.0
    assert _required(w, edit=speed_without_range) == 0

    def huge(s, ws, p):  # 4096^3 regions
        ws.grid[0] = ws.grid[1] = ws.grid[2] = 4096
    assert _required(w, edit=huge) == 0

    def fine_axis(n_sub):
        def edit(s, ws, p):  # one axis of 4096 cells x n_sub sub-cells, the others 1 x 1
            ws.grid[0], ws.grid[1], ws.grid[2] = 4096, 1, 1
            ws.sub[0], ws.sub[1], ws.sub[2] = n_sub, 1, 1
        return edit
    # at most 2^22 fine cells along an axis (the device's exact cell floor)
    assert _required(w, edit=fine_axis(1024)) > 0
    assert _required(w, edit=fine_axis(2048)) == 0

    def quad_massless(s, ws, p):
        s.phys[0] = 0.0
    assert _required(W.c3(0)) > 0 and _required(W.c3(0), edit=quad_massless) == 0


def test_arena_grows_by_the_per_node_rows():
    """Doubling t_e adds the per-node rows of the tree and the per-sample
    scratch: for the 6D Dubins airplane 191 bytes a node (state 24,
    control 12, parent, region, sub-region, claim check, accept list and
    V_E list 4 each, steps, set flag and sample flags 1 each, the kept end
    state 32, network features 64 and outputs 32), up to 256-byte
    alignment of each array."""
    from paper_2409_06807_gb300 import workloads as W
    a = _required(W.c2(0).with_(t_e=1 << 20))
    b = _required(W.c2(0).with_(t_e=1 << 21))
    assert a % 256 == 0 and b % 256 == 0
    assert abs((b - a) - 191 * (1 << 20)) <= 256 * 32
    q = _required(W.c3(0).with_(t_e=1 << 20))
    q2 = _required(W.c3(0).with_(t_e=1 << 21))
    # 12D: state 48, control 16, kept end state 64
    assert abs((q2 - q) - (191 + 24 + 4 + 32) * (1 << 20)) <= 256 * 32


def test_arena_one_byte_short_is_refused_before_any_device_work():
    """Failure injection on the host: an arena one byte smaller than
    kp_required_bytes makes kp_create return KP_ERR_OOM and leave *out NULL,
    a network arena one byte short makes kp_mlp_create do the same, and a
    server pool below its control area makes kp_server_create do the same.
    The arena pointer given is an aligned address nothing backs: the size
    check comes before any device call, so no GPU is needed and nothing is
    touched."""
    import ctypes as C
    from paper_2409_06807_gb300 import planner
    from paper_2409_06807_gb300 import workloads as W
    L = planner.lib()
    fake = C.c_void_p(1 << 20)  # 256-byte aligned, never dereferenced
    for w in (W.c1(0), W.c2(0), W.c3(0)):
        s, ws, p = planner.structs(w)
        need = L.kp_required_bytes(C.byref(s), C.byref(ws), len(w.boxes), C.byref(p))
        boxes = w.boxes.astype(np.float32).reshape(-1)
        obs = planner.Obstacles(boxes.ctypes.data_as(C.POINTER(C.c_float)), len(w.boxes))
        out = C.c_void_p(12345)
        st = L.kp_create(C.byref(s), C.byref(ws), C.byref(obs), C.byref(p), fake, need - 1,
                         None, C.byref(out))
        assert st == planner.ERR_OOM and out.value is None
        # misaligned arena: an argument error, also before any device call
        st = L.kp_create(C.byref(s), C.byref(ws), C.byref(obs), C.byref(p),
                         C.c_void_p((1 << 20) + 16), need, None, C.byref(out))
        assert st == planner.ERR_ARG and out.value is None
    m_need = L.kp_mlp_required_bytes(4096)
    params = np.zeros(L.kp_mlp_num_params(), np.float32)
    out = C.c_void_p(12345)
    st = L.kp_mlp_create(fake, m_need - 1, 4096, params.ctypes.data_as(C.POINTER(C.c_float)),
                         None, C.byref(out))
    assert st == planner.ERR_OOM and out.value is None

    class Cfg(C.Structure):
        _fields_ = [("team_blocks", C.c_int32), ("max_slots", C.c_int32), ("idle_ms", C.c_double)]
    c = Cfg(16, 64, 50.0)
    ctl = L.kp_server_required_bytes(64)
    out = C.c_void_p(12345)
    st = L.kp_server_create(C.byref(c), fake, ctl - 1, None, C.byref(out))
    assert st == planner.ERR_OOM and out.value is None
