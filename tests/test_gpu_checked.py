"""The lock-step suites on the bounds-checked build of the library.

With KP_CHECK defined, every array index the loop kernel derives is checked
against its array (node ids, sample keys, regions, sub-regions, V_E
positions, accepted-sample slots, block slots, broad-phase cells, box lists
and box ids); an index out of range records its site, is replaced by 0 (no
access leaves its array, nothing traps) and the call fails with that site.
The tiny and double-integrator lock-step suites, the one-block refill path
and the full-size frontiers run on that build in a process of their own, so
every pass they compare also shows that no index left its array."""
import os
import subprocess
import sys

import pytest

from paper_2409_06807_gb300 import workloads as W

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bounds_check_reports_an_index_past_the_tree():
    """The checked path itself: an index one past the tree, looked up
    through it, is reported with its site and read as element 0; the normal
    build refuses the self test without launching anything."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_2409_06807_gb300.build import build_planner\n"
        "from paper_2409_06807_gb300 import planner as P, workloads as W\n"
        "P.use_library(build_planner(check=True))\n"
        "assert P.lib().kp_bounds_checked() == 1\n"
        "g = P.Planner(W.tiny(W.DI))\n"
        "assert g.selftest_bounds() == P.ERR_CUDA, g.last_error()\n"
        "assert 'site 97' in g.last_error(), g.last_error()\n"
        "print('checked ok')\n" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0 and "checked ok" in r.stdout, r.stdout + r.stderr
    from paper_2409_06807_gb300.build import build_planner
    build_planner()
    from paper_2409_06807_gb300 import planner as P
    assert P.lib().kp_bounds_checked() == 0
    g = P.Planner(W.tiny(W.DI))
    assert g.selftest_bounds() == P.ERR_STATE


def test_lockstep_suites_on_the_bounds_checked_build():
    env = dict(os.environ, KP_TEST_BOUNDS_CHECKED="1")
    sel = ("lockstep_tiny or lockstep_c1 or refill_path or frontier_c2_full_shape "
           "or frontier_c3_quadrotor or plan_c1")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests",
                                                                     "test_gpu_parity.py"),
                        "-m", "gpu", "-q", "-x", "-p", "no:cacheprovider", "-k", sel],
                       capture_output=True, text=True, env=env, cwd=ROOT, timeout=1800)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout and "failed" not in r.stdout, tail
