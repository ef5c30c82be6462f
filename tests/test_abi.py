"""The C-ABI boundary without a GPU: the planner library builds for sm_103a,
loads, and exports (unmangled) every function that include/kp.h declares;
the Python binding types exactly those names; host-only size queries agree
with the binding's own constants.  No call here launches device work."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kp.h")


def _declared():
    """Function names declared at file scope in kp.h (comments stripped)."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    names = re.findall(r"^[A-Za-z_][\w \t\*]*?\b(kp_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2409_06807_gb300.build import build_planner
    return build_planner()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("kp_create", "kp_set_obstacles", "kp_reset", "kp_expand_step", "kp_plan",
                     "kp_plan_async", "kp_plan_result", "kp_export_tree", "kp_destroy"):
        assert required in names
    assert len(names) >= 30


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    L = C.CDLL(lib_path)
    for n in _declared():
        assert getattr(L, n) is not None


def test_binding_covers_the_header(lib_path):
    from paper_2409_06807_gb300 import planner
    assert sorted(planner.SIGNATURES) == _declared()


def test_host_size_queries(lib_path):
    from paper_2409_06807_gb300 import mlp, planner
    from paper_2409_06807_gb300 import workloads as W
    L = planner.lib()
    assert L.kp_mlp_num_params() == (mlp.N_H * (mlp.N_IN + 1) + mlp.N_H * (mlp.N_H + 1)
                                     + mlp.N_OUT * (mlp.N_H + 1))
    assert L.kp_mlp_required_bytes(4096) > L.kp_mlp_required_bytes(64) > 0
    assert L.kp_server_required_bytes(1024) >= L.kp_server_required_bytes(16) > 0
    w = W.c2(0)
    s, ws, p = planner.structs(w)
    a = L.kp_required_bytes(C.byref(s), C.byref(ws), len(w.boxes), C.byref(p))
    assert a > 0 and a % 256 == 0
