"""The planner library's host logic on CPU (no GPU): the broad-phase grid of
the step-hull test, the kd-tree of the free-space-obeying decomposition
(Sec. IV-B) and the query server's device-pool allocator.

The library's host driver is compiled into a small harness
(tests/host/kp_host_harness.cu) whose entry points call these parts
directly.  The grid's cell lists must give the verdict of testing every box
(a box meeting a hull is listed in a cell the hull touches), its shape must
follow the obstacle set, the kd-tree's leaves must be the oracle's, built
by the oracle's own code from the same rule, and the allocator must tile
the pool exactly with first-fit placement."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.kpo import Oracle
from paper_2409_06807_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host", "kp_host_harness.cu")
OUT = os.path.join(ROOT, "tests", "host", "_build", "libkphost.so")
CSRC = os.path.join(ROOT, "paper_2409_06807_gb300", "csrc")
LO, HI = np.zeros(3, np.float32), np.ones(3, np.float32)


def _stale():
    if not os.path.exists(OUT):
        return True
    deps = [SRC, os.path.join(ROOT, "include", "kp.h")] + \
        [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    return any(os.path.getmtime(p) > os.path.getmtime(OUT) for p in deps)


@pytest.fixture(scope="module")
def H():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc is needed to build the host harness")
    if _stale():
        os.makedirs(os.path.dirname(OUT), exist_ok=True)
        tmp = OUT + f".tmp{os.getpid()}"
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                        "-Xcompiler", "-fPIC", "-shared", "-I", os.path.join(ROOT, "include"),
                        "-o", tmp, SRC, "-cudart", "static"], check=True)
        os.replace(tmp, OUT)
    L = C.CDLL(OUT)
    f32 = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
    u8 = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
    i32 = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    L.kpt_blob.restype = C.c_int
    L.kpt_blob.argtypes = [f32, C.c_int, f32, f32, C.c_int, u8, i32, f32,
                           C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.kpt_blob_bytes.restype = C.c_int
    L.kpt_blob_bytes.argtypes = []
    L.kpt_kd_leaves.restype = C.c_int
    L.kpt_kd_leaves.argtypes = [f32, C.c_int, f32, f32, f32, C.c_int]
    u64 = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
    L.kpt_pool_new.restype = C.c_void_p
    L.kpt_pool_new.argtypes = [C.c_size_t]
    L.kpt_pool_alloc.restype = C.c_int
    L.kpt_pool_alloc.argtypes = [C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)]
    L.kpt_pool_free.argtypes = [C.c_void_p, C.c_size_t, C.c_size_t]
    L.kpt_pool_blocks.restype = C.c_int
    L.kpt_pool_blocks.argtypes = [C.c_void_p, u64, u64, C.c_int]
    L.kpt_pool_delete.argtypes = [C.c_void_p]
    return L


def blob(H, boxes, max_bytes=None):
    if max_bytes is None:
        max_bytes = H.kpt_blob_bytes()  # the arena's room for the blob
    boxes = np.ascontiguousarray(boxes, np.float32).reshape(-1, 6)
    buf = np.zeros(max(max_bytes, 16), np.uint8)
    g = np.zeros(3, np.int32)
    scale = np.zeros(3, np.float32)
    so, io, co = C.c_int(), C.c_int(), C.c_int()
    n = H.kpt_blob(boxes if len(boxes) else np.zeros((1, 6), np.float32), len(boxes), LO, HI,
                   max_bytes, buf, g, scale, C.byref(so), C.byref(io), C.byref(co))
    C_ = int(np.prod(g))
    start = buf[so.value:so.value + 2 * (C_ + 1)].view(np.uint16).astype(np.int64)
    ids = buf[io.value:io.value + 2 * int(start[-1])].view(np.uint16).astype(np.int64)
    clear = buf[co.value:co.value + C_].copy() if co.value >= 0 else None
    return dict(bytes=n, g=g.tolist(), scale=scale, start=start, ids=ids, clear=clear)


def cell(v, a, bp):
    """The builder's cell of coordinate v on axis a, in float32."""
    t = np.float32(np.float32(v) - LO[a]) * bp["scale"][a]
    g = bp["g"][a]
    return np.where(t >= 0, np.where(t < np.float32(g), np.floor(t).astype(np.int64), g - 1), 0)


def listed(bp, h):
    """Box ids listed in the cells that hull h (lo xyz, hi xyz) touches."""
    r = [(int(cell(h[a], a, bp)), int(cell(h[3 + a], a, bp))) for a in range(3)]
    gx, gy, _ = bp["g"]
    out = set()
    for z in range(r[2][0], r[2][1] + 1):
        for y in range(r[1][0], r[1][1] + 1):
            for x in range(r[0][0], r[0][1] + 1):
                c = x + gx * (y + gy * z)
                out.update(bp["ids"][bp["start"][c]:bp["start"][c + 1]].tolist())
    return out


def hulls(rng, n, size):
    p = rng.uniform(-0.02, 1.02, (n, 3)).astype(np.float32)
    d = rng.uniform(-size, size, (n, 3)).astype(np.float32)
    return np.concatenate([np.minimum(p, p + d), np.maximum(p, p + d)], 1).astype(np.float32)


def turned(boxes, order):
    return np.ascontiguousarray(np.concatenate([boxes[:, list(order)],
                                                boxes[:, [3 + a for a in order]]], 1))


def layouts():
    big = np.random.default_rng(7)
    lo = big.uniform(0.0, 0.45, (400, 3)).astype(np.float32)
    large = np.concatenate([lo, lo + big.uniform(0.3, 0.5, (400, 3)).astype(np.float32)], 1)
    return {"forest": W.c2(0).boxes, "building": W.c3(0).boxes, "random": W.c1(3).boxes,
            "forest along x": turned(W.c2(0).boxes, (2, 0, 1)),
            "forest along y": turned(W.c2(0).boxes, (0, 2, 1)), "large boxes": large,
            "most boxes": W.random_boxes(9, 4096, side=(0.005, 0.03))}


def test_grid_shape_follows_the_obstacles(H):
    shapes = {k: blob(H, b)["g"] for k, b in layouts().items()}
    assert shapes["forest"] == [64, 64, 1]
    assert shapes["forest along x"] == [1, 64, 64]
    assert shapes["forest along y"] == [64, 1, 64]
    assert shapes["building"] == [16, 16, 16]
    # too many (cell, box) entries for any 4096-cell shape: an isotropic
    # coarser grid
    g = shapes["large boxes"]
    assert g[0] == g[1] == g[2] < 16
    assert blob(H, np.zeros((0, 6), np.float32))["g"] == [1, 1, 1]


@pytest.mark.parametrize("name", ["forest", "building", "random", "forest along x", "large boxes",
                                  "most boxes"])
def test_cell_lists_give_the_verdict_of_every_box(H, name):
    """Every box meeting a hull is listed in a cell the hull touches; the
    blob fits the arena's room for it (KP_BLOB_BYTES) even at the box
    capacity of 4,096."""
    boxes = layouts()[name]
    bp = blob(H, boxes)
    n = len(boxes)
    assert bp["bytes"] <= H.kpt_blob_bytes()
    assert np.all(np.diff(bp["start"]) >= 0) and np.all(bp["ids"] < n)
    # each box is listed once in every cell of its range, nowhere else
    want = sum(np.prod([int(cell(b[3 + a], a, bp)) - int(cell(b[a], a, bp)) + 1 for a in range(3)])
               for b in boxes)
    assert len(bp["ids"]) == want
    rng = np.random.default_rng(11)
    for size in (0.01, 0.08):
        for h in hulls(rng, 400, size):
            meets = np.flatnonzero(np.all(boxes[:, :3] <= h[3:], 1) & np.all(h[:3] <= boxes[:, 3:], 1))
            assert set(meets.tolist()) <= listed(bp, h)


def clear_by_cell(bp, h):
    """The device's clearance test of hull h in float32: inside the cell of
    its low corner grown by that cell's clearance on every side."""
    t = [(np.float32(np.float32(h[a]) - LO[a]) * bp["scale"][a],
          np.float32(np.float32(h[3 + a]) - LO[a]) * bp["scale"][a]) for a in range(3)]
    c0 = [int(cell(h[a], a, bp)) for a in range(3)]
    gx, gy, _ = bp["g"]
    r = np.float32(bp["clear"][c0[0] + gx * (c0[1] + gy * c0[2])]) * np.float32(0.0625)
    return bool(r > 0 and all(t[a][0] >= np.float32(c0[a]) - r and
                              t[a][1] <= np.float32(c0[a]) + np.float32(1.0) + r for a in range(3)))


@pytest.mark.parametrize("name", ["forest", "building", "random", "forest along y", "large boxes"])
def test_cell_clearance_never_hides_a_box(H, name):
    """A hull that the cell clearance declares free meets no box (every box
    tested, closed sets), on hulls scattered over the workspace and on hulls
    that graze the boxes' faces; and the clearance does declare most hulls
    away from the obstacles free.  The clearances equal the ones the
    oracle's work count computes from the same rule in its own code."""
    boxes = layouts()[name]
    bp = blob(H, boxes)
    assert bp["clear"] is not None
    rng = np.random.default_rng(13)
    free = tested = 0
    grazing = []
    for b in boxes[rng.integers(0, len(boxes), 300)]:
        a = int(rng.integers(0, 3))
        side = int(rng.integers(0, 2))
        p = rng.uniform(b[:3], b[3:]).astype(np.float32)
        p[a] = b[3 * side + a] + np.float32((2 * side - 1) * rng.uniform(0.0, 0.02))
        d = rng.uniform(-0.004, 0.004, 3).astype(np.float32)
        grazing.append(np.concatenate([np.minimum(p, p + d), np.maximum(p, p + d)]))
    for h in list(hulls(rng, 3000, 0.006)) + grazing:
        if clear_by_cell(bp, h):
            free += 1
            meets = np.all(boxes[:, :3] <= h[3:], 1) & np.all(h[:3] <= boxes[:, 3:], 1)
            assert not meets.any(), (h, np.flatnonzero(meets)[:3])
        tested += 1
    if name != "large boxes":
        assert free > 0.3 * tested, (free, tested)
    o = Oracle(W.tiny(W.DI, seed=0, n_boxes=0).with_(boxes=np.ascontiguousarray(boxes)))
    o.set_work_grid(bp["g"])
    np.testing.assert_array_equal(o.work_clearance(), bp["clear"].astype(np.int32))


def test_grid_respects_the_byte_budget(H):
    """A query whose blob must fit a small budget (a server slot) gets a
    coarser grid, never a larger blob."""
    boxes = W.c3(0).boxes
    full = blob(H, boxes)
    small = blob(H, boxes, max_bytes=49152)
    assert small["bytes"] <= 49152 < full["bytes"] or full["bytes"] <= 49152
    assert np.prod(small["g"]) <= np.prod(full["g"])


def leaves(H, boxes):
    boxes = np.ascontiguousarray(boxes, np.float32).reshape(-1, 6)
    out = np.zeros((16384, 6), np.float32)
    n = H.kpt_kd_leaves(boxes if len(boxes) else np.zeros((1, 6), np.float32), len(boxes),
                        LO, HI, out, 16384)
    return n, out[:max(n, 0)]


@pytest.mark.parametrize("name", ["forest", "random", "one box", "none"])
def test_kd_tree_leaves_are_the_oracles(H, name):
    boxes = {"forest": W.c2(0).boxes, "random": W.c1(3).boxes,
             "one box": np.array([[0.25, 0.25, 0.25, 0.75, 0.75, 0.75]], np.float32),
             "none": np.zeros((0, 6), np.float32)}[name]
    n, ours = leaves(H, boxes)
    lo, hi = Oracle(W.tiny(W.DI, seed=0, n_boxes=0).with_(boxes=boxes, fso=True)).fso_leaves()
    assert n == len(lo)
    np.testing.assert_array_equal(ours[:, :3], lo.astype(np.float32))
    np.testing.assert_array_equal(ours[:, 3:], hi.astype(np.float32))


def _free_blocks(H, s):
    offs = np.zeros(4096, np.uint64)
    sizes = np.zeros(4096, np.uint64)
    n = H.kpt_pool_blocks(s, offs, sizes, 4096)
    assert n <= 4096
    return [(int(o), int(z)) for o, z in zip(offs[:n], sizes[:n])]


def test_server_pool_allocator(H):
    """The server admits a query when its arena fits the device pool: first
    fit over the free list in 256-byte granules, coalescing neighbours on
    free.  A seeded mix of allocations and frees keeps the free list sorted,
    aligned and coalesced, free plus allocated tiling the pool exactly, and
    every allocation at the lowest free block that fits."""
    total = 64 << 20
    s = H.kpt_pool_new(total)
    rng = np.random.default_rng(5)
    live = {}
    try:
        for step in range(3000):
            before = _free_blocks(H, s)
            if live and (rng.random() < 0.45 or len(live) > 60):
                off = int(rng.choice(sorted(live)))
                H.kpt_pool_free(s, off, live.pop(off))
            else:
                want = int(rng.integers(1, 3 << 20))
                need = (want + 255) // 256 * 256
                off = C.c_size_t()
                ok = H.kpt_pool_alloc(s, want, C.byref(off))
                fits = [o for o, z in before if z >= need]
                assert bool(ok) == bool(fits)
                if ok:
                    assert off.value == fits[0]
                    live[off.value] = want
            free = _free_blocks(H, s)
            assert all(o % 256 == 0 and z % 256 == 0 and z > 0 for o, z in free)
            assert all(a[0] + a[1] < b[0] for a, b in zip(free, free[1:]))  # sorted, coalesced
            spans = sorted(free + [(o, (z + 255) // 256 * 256) for o, z in live.items()])
            pos = 0
            for o, z in spans:
                assert o == pos
                pos += z
            assert pos == total
        for off in list(live):
            H.kpt_pool_free(s, off, live.pop(off))
        assert _free_blocks(H, s) == [(0, total)]
    finally:
        H.kpt_pool_delete(s)
