"""Builds the FP64 CPU oracle into ``oracle/libkpo.so``.

Test infrastructure only: the oracle checks the CUDA implementation and is
never part of the product path.  Compiled with ``-ffp-contract=off`` so that
no multiply-add is fused: Eq. 3-5 then round exactly as written, which the
device code reproduces with explicitly rounded double operations.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["philox.c", "model.c", "planner.c", "mlp.c", "work.c"]
LIB = os.path.join(HERE, "libkpo.so")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = SOURCES + ["kpo.h", "kpo_internal.h"]
    return any(os.path.getmtime(os.path.join(HERE, s)) > t for s in deps)


def compile_oracle(src_dir: str, out: str) -> str:
    """Compile the oracle sources found in src_dir into the library 'out'."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-Wall", "-Wextra", "-Wno-unused-parameter",
           "-o", tmp] + [os.path.join(src_dir, s) for s in SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build_oracle(force: bool = False) -> str:
    """Compile the oracle shared library if needed; returns its path."""
    if force or _stale():
        compile_oracle(HERE, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
