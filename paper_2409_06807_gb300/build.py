"""Builds the CUDA planner library ``libkinopax.so`` in-tree, for sm_103a.

The translation units compile in parallel (one per system plus the host
driver) and link into one shared library with the CUDA runtime statically
linked, so the library only needs the driver at run time.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libkinopax.so")
ROOT = os.path.dirname(HERE)
UNITS = ["kp_api.cu", "kp_sys_di.cu", "kp_sys_dubins.cu", "kp_sys_quad.cu", "kp_mlp.cu", "kp_server.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the planner")
    return path


def _deps():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    out.append(os.path.join(ROOT, "include", "kp.h"))
    return out


LIB_CHECK = os.path.join(HERE, "libkinopax_check.so")


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _deps())


def _compile(unit: str, extra, build_dir: str = BUILD) -> str:
    obj = os.path.join(build_dir, unit.replace(".cu", ".o"))
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-I", os.path.join(ROOT, "include"), "-c", os.path.join(CSRC, unit), "-o", obj,
           *extra]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {unit}:\n{r.stdout}\n{r.stderr}")
    return obj


def build_planner(force: bool = False, verbose_ptxas: bool = False, check: bool = False) -> str:
    """Compile the planner library if any source changed; returns its path.
    check=True builds the bounds-checked variant (KP_CHECK defined: every
    array index the loop kernel derives is checked, see include/kp.h) into
    its own library, libkinopax_check.so."""
    lib, build_dir = (LIB_CHECK, BUILD + "_check") if check else (LIB, BUILD)
    if not force and not _stale(lib):
        return lib
    os.makedirs(build_dir, exist_ok=True)
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    if check:
        extra = extra + ["-DKP_CHECK"]
    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(lambda u: _compile(u, extra, build_dir), UNITS))
    tmp = lib + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build_planner(force=True, verbose_ptxas="-v" in sys.argv))
