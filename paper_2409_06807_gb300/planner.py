"""Thin ctypes binding of the C ABI in ``include/kp.h``.

Argument marshalling only: every step of the planner runs in the CUDA
library ``libkinopax.so``.  PyTorch supplies the device arena (a uint8 CUDA
tensor) and the stream.  There is no CPU fallback: constructing a
``Planner`` without the compiled library or without a CUDA device raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .workloads import STATE_DIM, CONTROL_DIM

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkinopax.so")

OK, NO_SOLUTION, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_STATE = 0, 1, -1, -2, -3, -4, -5
STATUS_NAMES = {0: "OK", 1: "NO_SOLUTION", -1: "ERR_ARG", -2: "ERR_OOM", -3: "ERR_CUDA",
                -4: "ERR_TIMEOUT", -5: "ERR_STATE"}
MAX_BOXES = 4096


class KpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class System(C.Structure):
    _fields_ = [("id", C.c_int32), ("dt", C.c_float), ("k_min", C.c_int32),
                ("k_max", C.c_int32), ("x_lo", C.c_float * 12), ("x_hi", C.c_float * 12),
                ("u_lo", C.c_float * 4), ("u_hi", C.c_float * 4), ("phys", C.c_float * 16)]


class Workspace(C.Structure):
    _fields_ = [("lo", C.c_float * 3), ("hi", C.c_float * 3), ("grid", C.c_int32 * 3),
                ("speed_bins", C.c_int32), ("speed_hi", C.c_float), ("sub", C.c_int32 * 3),
                ("state_grid", C.c_int32 * 12), ("fso", C.c_int32)]


class Obstacles(C.Structure):
    _fields_ = [("boxes", C.POINTER(C.c_float)), ("n_boxes", C.c_int32)]


class Goal(C.Structure):
    _fields_ = [("center", C.c_float * 3), ("radius", C.c_float)]


class Params(C.Structure):
    _fields_ = [("t_e", C.c_int32), ("lambda_max", C.c_int32), ("delta", C.c_double),
                ("eps", C.c_double), ("seed", C.c_uint64)]


class Budget(C.Structure):
    _fields_ = [("max_iters", C.c_int32), ("max_ms", C.c_double)]


class Traj(C.Structure):
    _fields_ = [("capacity", C.c_int32), ("n_edges", C.c_int32),
                ("states", C.POINTER(C.c_float)), ("ctrls", C.POINTER(C.c_float)),
                ("steps", C.POINTER(C.c_int32))]


STAT_FIELDS = ("iteration", "n_ve", "lambda", "n_samples", "n_valid", "n_accepted",
               "n_nodes", "goal_node")


class IterStats(C.Structure):
    _fields_ = [(n if n != "lambda" else "lambda_", C.c_int32) for n in STAT_FIELDS] + \
        [("phase_ns", C.c_int32 * 12)]


class Info(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("n_nodes", "n_ve", "iteration", "goal_node", "state",
                                           "n_regions", "n_subregions", "state_dim",
                                           "control_dim", "n_boxes", "grid_blocks")] + \
        [(n, C.c_int64) for n in ("n_samples", "n_steps", "n_hull_checks", "n_box_tests")] + \
        [("bp_cells", C.c_int32), ("bp_grid", C.c_int32 * 3),
         ("n_key_batches", C.c_int64), ("n_lane_refills", C.c_int64)]


class TreeView(C.Structure):
    _fields_ = [("capacity", C.c_int32), ("n_nodes", C.c_int32), ("iteration", C.c_int32),
                ("state", C.c_void_p), ("parent", C.c_void_p), ("ctrl", C.c_void_p),
                ("steps", C.c_void_p), ("region", C.c_void_p), ("sub", C.c_void_p),
                ("in_ve", C.c_void_p), ("n_valid", C.c_void_p), ("n_invalid", C.c_void_p),
                ("cov", C.c_void_p), ("avail", C.c_void_p), ("thr", C.c_void_p),
                ("visited", C.c_void_p)]


class SampleLog(C.Structure):
    _fields_ = [("capacity", C.c_int32)] + [(n, C.c_void_p) for n in (
        "node", "k", "uraw", "flags", "fail_step", "region", "sub", "state")]


_lib = None
_lib_path = LIB_PATH

# every entry point of include/kp.h: name -> (restype, argtypes)
_vp = C.c_void_p
SIGNATURES = {
    "kp_required_bytes": (C.c_size_t, [C.POINTER(System), C.POINTER(Workspace), C.c_int32,
                                       C.POINTER(Params)]),
    "kp_create": (C.c_int, [C.POINTER(System), C.POINTER(Workspace), C.POINTER(Obstacles),
                            C.POINTER(Params), _vp, C.c_size_t, _vp, C.POINTER(_vp)]),
    "kp_set_obstacles": (C.c_int, [_vp, C.POINTER(Obstacles)]),
    "kp_reset": (C.c_int, [_vp, C.POINTER(C.c_float), C.POINTER(Goal), C.c_uint64]),
    "kp_expand_step": (C.c_int, [_vp, C.c_int32, C.POINTER(IterStats), C.POINTER(C.c_int32)]),
    "kp_plan": (C.c_int, [_vp, C.POINTER(C.c_float), C.POINTER(Goal), C.POINTER(Budget),
                          C.POINTER(Traj)]),
    "kp_plan_async": (C.c_int, [_vp, C.POINTER(C.c_float), C.POINTER(Goal), C.POINTER(Budget),
                                C.c_int32]),
    "kp_plan_result": (C.c_int, [_vp, C.POINTER(Traj)]),
    "kp_last_launch_ms": (C.c_int, [_vp, C.POINTER(C.c_float)]),
    "kp_get_info": (C.c_int, [_vp, C.POINTER(Info)]),
    "kp_export_tree": (C.c_int, [_vp, C.POINTER(TreeView)]),
    "kp_import_tree": (C.c_int, [_vp, C.POINTER(TreeView)]),
    "kp_grow": (C.c_int, [_vp, _vp, C.c_size_t, C.c_int32]),
    "kp_resume": (C.c_int, [_vp, C.POINTER(Budget), C.POINTER(Traj)]),
    "kp_set_sample_log": (C.c_int, [_vp, C.POINTER(SampleLog)]),
    "kp_set_wait_limit": (C.c_int, [_vp, C.c_uint64]),
    "kp_set_grid_limit": (C.c_int, [_vp, C.c_int32]),
    "kp_set_extract_ids": (C.c_int, [_vp, C.c_int32]),
    "kp_selftest_wait_timeout": (C.c_int, [_vp]),
    "kp_bounds_checked": (C.c_int32, []),
    "kp_selftest_bounds": (C.c_int, [_vp]),
    "kp_plan_static": (C.c_int, [C.POINTER(System), C.POINTER(Workspace), C.POINTER(Obstacles),
                                 C.POINTER(Params), C.POINTER(C.c_float), C.POINTER(Goal),
                                 C.POINTER(Budget), C.POINTER(Traj), _vp]),
    "kp_measure_lane_peak": (C.c_int, [_vp, C.POINTER(C.c_double)]),
    "kp_mlp_num_params": (C.c_int32, []),
    "kp_mlp_required_bytes": (C.c_size_t, [C.c_int32]),
    "kp_mlp_create": (C.c_int, [_vp, C.c_size_t, C.c_int32, C.POINTER(C.c_float), _vp,
                                C.POINTER(_vp)]),
    "kp_mlp_set_params": (C.c_int, [_vp, C.POINTER(C.c_float)]),
    "kp_mlp_get_params": (C.c_int, [_vp, C.POINTER(C.c_float)]),
    "kp_mlp_forward": (C.c_int, [_vp, _vp, C.c_int32, _vp]),
    "kp_mlp_gradients": (C.c_int, [_vp, _vp, _vp, C.c_int32, C.POINTER(C.c_float),
                                   C.POINTER(C.c_float)]),
    "kp_mlp_train_step": (C.c_int, [_vp, _vp, _vp, C.c_int32, C.c_float, C.POINTER(C.c_float)]),
    "kp_mlp_train_epoch": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int64, C.c_float,
                                     C.POINTER(C.c_float)]),
    "kp_mlp_destroy": (None, [_vp]),
    "kp_attach_mlp": (C.c_int, [_vp, _vp, C.c_float]),
    "kp_set_harvest": (C.c_int, [_vp, _vp, _vp, C.c_int32, _vp]),
    "kp_server_required_bytes": (C.c_size_t, [C.c_int32]),
    "kp_server_create": (C.c_int, [C.c_void_p, _vp, C.c_size_t, _vp, C.POINTER(_vp)]),
    "kp_server_submit": (C.c_int, [_vp, C.POINTER(System), C.POINTER(Workspace),
                                   C.POINTER(Obstacles), C.POINTER(Params), C.POINTER(C.c_float),
                                   C.POINTER(Goal), C.POINTER(Budget), C.POINTER(C.c_int64)]),
    "kp_server_poll": (C.c_int, [_vp, C.c_void_p, C.c_int32, C.POINTER(C.c_int32)]),
    "kp_server_result": (C.c_int, [_vp, C.c_int64, C.POINTER(Traj)]),
    "kp_server_stats_get": (C.c_int, [_vp, C.c_void_p]),
    "kp_server_destroy": (None, [_vp]),
    "kp_last_error": (C.c_char_p, [_vp]),
    "kp_destroy": (None, [_vp]),
}


def use_library(path):
    """Selects the planner library later calls use (for example the
    bounds-checked build of build.build_planner(check=True)); contexts made
    with another library must be closed first."""
    global _lib, _lib_path
    _lib, _lib_path = None, path


def lib():
    """The loaded planner library.  Raises when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_lib_path):
            raise RuntimeError(
                f"CUDA planner library missing ({_lib_path}); build it with "
                "paper_2409_06807_gb300.build.build_planner()")
        L = C.CDLL(_lib_path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _fptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def structs(w):
    """C structs of a workload (float32 values taken as they are)."""
    s = System()
    s.id = w.system
    s.dt = float(w.dt)
    s.k_min, s.k_max = int(w.k_min), int(w.k_max)
    for i in range(12):
        s.x_lo[i] = float(w.x_lo[i])
        s.x_hi[i] = float(w.x_hi[i])
    for i in range(4):
        s.u_lo[i] = float(w.u_lo[i])
        s.u_hi[i] = float(w.u_hi[i])
    for i in range(16):
        s.phys[i] = float(w.phys[i])
    ws = Workspace()
    for a in range(3):
        ws.lo[a] = float(w.ws_lo[a])
        ws.hi[a] = float(w.ws_hi[a])
        ws.grid[a] = int(w.grid[a])
        ws.sub[a] = int(w.sub[a])
    ws.speed_bins = int(w.speed_bins)
    for i in range(12):
        ws.state_grid[i] = int(w.state_grid[i])
    ws.fso = 1 if getattr(w, "fso", False) else 0
    ws.speed_hi = float(w.speed_hi)
    p = Params()
    p.t_e, p.lambda_max = int(w.t_e), int(w.lambda_max)
    p.delta, p.eps = float(w.delta), float(w.eps)
    p.seed = int(w.seed) & 0xFFFFFFFFFFFFFFFF
    return s, ws, p


def measure_lane_peak(stream=None):
    """Measured lane-issue peak of the current device (lane operations per
    second) from the library's FMA microbenchmark (kp_measure_lane_peak)."""
    out = C.c_double()
    st = lib().kp_measure_lane_peak(C.c_void_p(stream.cuda_stream if stream is not None else 0),
                                    C.byref(out))
    if st != OK:
        raise KpError(st, "kp_measure_lane_peak failed")
    return out.value


def goal_struct(w):
    g = Goal()
    for a in range(3):
        g.center[a] = float(w.goal_c[a])
    g.radius = float(w.goal_r)
    return g


class Planner:
    """One planning context on one CUDA device (see include/kp.h)."""

    def __init__(self, w, device=None, stream=None, box_capacity=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the planner needs a CUDA device")
        L = lib()
        self.w = w
        self.d = STATE_DIM[w.system]
        self.n_ctrl = CONTROL_DIM[w.system]
        self.device = (torch.device("cuda", torch.cuda.current_device()) if device is None
                       else torch.device(device))
        self._sys, self._ws, self._prm = structs(w)
        cap = int(box_capacity if box_capacity is not None else len(w.boxes))
        self.box_capacity = cap
        nbytes = L.kp_required_bytes(C.byref(self._sys), C.byref(self._ws), cap,
                                     C.byref(self._prm))
        if nbytes == 0:
            raise KpError(ERR_ARG, "invalid workload")
        with torch.cuda.device(self.device):
            self.arena = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.arena_bytes = int(nbytes)
        boxes = np.ascontiguousarray(np.asarray(w.boxes, np.float32).reshape(-1, 6))
        obs = Obstacles(_fptr(boxes) if len(boxes) else None, len(boxes))
        self._ctx = C.c_void_p()
        st = L.kp_create(C.byref(self._sys), C.byref(self._ws), C.byref(obs),
                         C.byref(self._prm), C.c_void_p(self.arena.data_ptr()),
                         self.arena_bytes, C.c_void_p(self.stream.cuda_stream),
                         C.byref(self._ctx))
        if st != OK:
            raise KpError(st, "kp_create failed")
        self._log = None
        info = self.info()
        self.n_regions, self.n_sub = info["n_regions"], info["n_subregions"]

    def close(self):
        if getattr(self, "_ctx", None):
            lib().kp_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st not in (OK, NO_SOLUTION):
            msg = lib().kp_last_error(self._ctx)
            raise KpError(st, f"{what}: {msg.decode() if msg else ''}")
        return st

    # ------------------------------------------------------------------
    def set_obstacles(self, boxes):
        boxes = np.ascontiguousarray(np.asarray(boxes, np.float32).reshape(-1, 6))
        obs = Obstacles(_fptr(boxes) if len(boxes) else None, len(boxes))
        self._check(lib().kp_set_obstacles(self._ctx, C.byref(obs)), "kp_set_obstacles")
        # a kd-tree decomposition has as many regions as the new set gives
        info = self.info()
        self.n_regions, self.n_sub = info["n_regions"], info["n_subregions"]

    def reset(self, x_init=None, goal=None, seed=None):
        w = self.w
        x = np.ascontiguousarray(w.x_init if x_init is None else x_init, np.float32)
        g = goal_struct(w) if goal is None else goal
        s = int(w.seed if seed is None else seed) & 0xFFFFFFFFFFFFFFFF
        return self._check(lib().kp_reset(self._ctx, _fptr(x), C.byref(g), s), "kp_reset")

    def expand_step(self, n_iters=1):
        out = (IterStats * n_iters)()
        n_run = C.c_int32()
        self._check(lib().kp_expand_step(self._ctx, n_iters, out, C.byref(n_run)),
                    "kp_expand_step")
        res = []
        for s in out[: n_run.value]:
            d = {f: getattr(s, f if f != "lambda" else "lambda_") for f in STAT_FIELDS}
            d["phase_ns"] = list(s.phase_ns)
            res.append(d)
        return res

    def plan(self, max_iters=1000, max_ms=0.0, capacity=4096, x_init=None, goal=None):
        w = self.w
        x = np.ascontiguousarray(w.x_init if x_init is None else x_init, np.float32)
        g = goal_struct(w) if goal is None else goal
        states = np.zeros((capacity, 12), np.float32)
        ctrls = np.zeros((capacity, 4), np.float32)
        steps = np.zeros(capacity, np.int32)
        t = Traj(capacity, 0, _fptr(states), _fptr(ctrls),
                 steps.ctypes.data_as(C.POINTER(C.c_int32)))
        b = Budget(int(max_iters), float(max_ms))
        st = self._check(lib().kp_plan(self._ctx, _fptr(x), C.byref(g), C.byref(b), C.byref(t)),
                         "kp_plan")
        n = t.n_edges
        return st, dict(states=states[:n, : self.d], ctrls=ctrls[:n, : self.n_ctrl],
                        steps=steps[:n])

    def grow(self, t_e):
        """Raises the node cap to t_e (Remark 1): a new arena, the tree and
        tables carried over by the device."""
        import torch
        L = lib()
        prm = Params()
        C.memmove(C.byref(prm), C.byref(self._prm), C.sizeof(Params))
        prm.t_e = int(t_e)
        nbytes = L.kp_required_bytes(C.byref(self._sys), C.byref(self._ws), self.box_capacity,
                                     C.byref(prm))
        if nbytes == 0:
            raise KpError(ERR_ARG, "invalid node cap")
        with torch.cuda.device(self.device):
            arena = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        self._check(L.kp_grow(self._ctx, C.c_void_p(arena.data_ptr()), int(nbytes), int(t_e)),
                    "kp_grow")
        self.arena, self.arena_bytes, self._prm = arena, int(nbytes), prm
        self.w = self.w.with_(t_e=int(t_e))

    def resume(self, max_iters=1000, max_ms=0.0, capacity=4096):
        """Continues planning from the current tree."""
        states = np.zeros((capacity, 12), np.float32)
        ctrls = np.zeros((capacity, 4), np.float32)
        steps = np.zeros(capacity, np.int32)
        t = Traj(capacity, 0, _fptr(states), _fptr(ctrls),
                 steps.ctypes.data_as(C.POINTER(C.c_int32)))
        b = Budget(int(max_iters), float(max_ms))
        st = self._check(lib().kp_resume(self._ctx, C.byref(b), C.byref(t)), "kp_resume")
        n = t.n_edges
        return st, dict(states=states[:n, : self.d], ctrls=ctrls[:n, : self.n_ctrl],
                        steps=steps[:n])

    def plan_adaptive(self, max_iters=1000, growth=2.0, t_e_max=1 << 24, capacity=4096):
        """Plans with the current node cap and, while the tree fills up
        without reaching the goal, grows the cap by 'growth' and continues
        (Remark 1).  Returns (status, trajectory, number of growths)."""
        st, traj = self.plan(max_iters=max_iters, capacity=capacity)
        grown = 0
        while st == NO_SOLUTION and self.info()["state"] == 2 and self.w.t_e < t_e_max:
            self.grow(min(int(self.w.t_e * growth), t_e_max))
            grown += 1
            left = max_iters - self.info()["iteration"]
            if left < 1:
                break
            st, traj = self.resume(max_iters=left, capacity=capacity)
        return st, traj, grown

    def plan_async(self, max_iters=1000, max_ms=0.0, capacity=4096, x_init=None, goal=None):
        """Enqueue a whole query on the stream; collect it with plan_result."""
        w = self.w
        x = np.ascontiguousarray(w.x_init if x_init is None else x_init, np.float32)
        g = goal_struct(w) if goal is None else goal
        b = Budget(int(max_iters), float(max_ms))
        self._check(lib().kp_plan_async(self._ctx, _fptr(x), C.byref(g), C.byref(b),
                                        int(capacity)), "kp_plan_async")
        self._pending_cap = int(capacity)

    def plan_result(self):
        cap = self._pending_cap
        states = np.zeros((cap, 12), np.float32)
        ctrls = np.zeros((cap, 4), np.float32)
        steps = np.zeros(cap, np.int32)
        t = Traj(cap, 0, _fptr(states), _fptr(ctrls),
                 steps.ctypes.data_as(C.POINTER(C.c_int32)))
        st = self._check(lib().kp_plan_result(self._ctx, C.byref(t)), "kp_plan_result")
        n = t.n_edges
        return st, dict(states=states[:n, : self.d], ctrls=ctrls[:n, : self.n_ctrl],
                        steps=steps[:n])

    def last_launch_ms(self):
        ms = C.c_float()
        self._check(lib().kp_last_launch_ms(self._ctx, C.byref(ms)), "kp_last_launch_ms")
        return ms.value

    def info(self):
        i = Info()
        self._check(lib().kp_get_info(self._ctx, C.byref(i)), "kp_get_info")
        return {f: (list(getattr(i, f)) if f == "bp_grid" else getattr(i, f))
                for f, _ in Info._fields_}

    # ------------------------------------------------------------------
    def export_tree(self):
        n = self.info()["n_nodes"]
        R, ns = self.n_regions, self.n_sub
        t = dict(state=np.zeros((n, 12), np.float32), parent=np.zeros(n, np.int32),
                 ctrl=np.zeros((n, 4), np.float32), steps=np.zeros(n, np.int32),
                 region=np.zeros(n, np.int32), sub=np.zeros(n, np.int32),
                 in_ve=np.zeros(n, np.uint8), n_valid=np.zeros(R, np.uint32),
                 n_invalid=np.zeros(R, np.uint32), cov=np.zeros(R, np.uint32),
                 avail=np.zeros(R, np.uint8), thr=np.zeros(R, np.uint64),
                 visited=np.zeros(ns, np.uint8))
        v = TreeView(n, 0, 0, *[t[k].ctypes.data for k in (
            "state", "parent", "ctrl", "steps", "region", "sub", "in_ve", "n_valid",
            "n_invalid", "cov", "avail", "thr", "visited")])
        self._check(lib().kp_export_tree(self._ctx, C.byref(v)), "kp_export_tree")
        t["state"] = t["state"][:, : self.d]
        t["ctrl"] = t["ctrl"][:, : self.n_ctrl]
        t["n_nodes"] = v.n_nodes
        t["iteration"] = v.iteration
        return t

    def import_tree(self, t):
        n = int(t["n_nodes"])
        st = np.zeros((n, 12), np.float32)
        st[:, : self.d] = np.asarray(t["state"], np.float32)[:n, : self.d]
        ct = np.zeros((n, 4), np.float32)
        ct[:, : self.n_ctrl] = np.asarray(t["ctrl"], np.float32)[:n, : self.n_ctrl]
        arrs = dict(state=st, parent=np.ascontiguousarray(t["parent"][:n], np.int32), ctrl=ct,
                    steps=np.ascontiguousarray(t["steps"][:n], np.int32),
                    region=np.ascontiguousarray(t["region"][:n], np.int32),
                    sub=np.ascontiguousarray(t["sub"][:n], np.int32),
                    in_ve=np.ascontiguousarray(t["in_ve"][:n], np.uint8),
                    n_valid=np.ascontiguousarray(t["n_valid"], np.uint32),
                    n_invalid=np.ascontiguousarray(t["n_invalid"], np.uint32),
                    thr=np.ascontiguousarray(t["thr"], np.uint64),
                    visited=np.ascontiguousarray(t["visited"], np.uint8))
        v = TreeView(n, n, int(t["iteration"]), arrs["state"].ctypes.data,
                     arrs["parent"].ctypes.data, arrs["ctrl"].ctypes.data,
                     arrs["steps"].ctypes.data, arrs["region"].ctypes.data,
                     arrs["sub"].ctypes.data, arrs["in_ve"].ctypes.data,
                     arrs["n_valid"].ctypes.data, arrs["n_invalid"].ctypes.data, None, None,
                     arrs["thr"].ctypes.data, arrs["visited"].ctypes.data)
        self._check(lib().kp_import_tree(self._ctx, C.byref(v)), "kp_import_tree")

    # ------------------------------------------------------------------
    def enable_log(self, capacity):
        import torch
        dev = self.device
        self._log = dict(
            node=torch.zeros(capacity, dtype=torch.int32, device=dev),
            k=torch.zeros(capacity, dtype=torch.int32, device=dev),
            uraw=torch.zeros(capacity * 4, dtype=torch.int32, device=dev),
            flags=torch.zeros(capacity, dtype=torch.uint8, device=dev),
            fail_step=torch.zeros(capacity, dtype=torch.int32, device=dev),
            region=torch.zeros(capacity, dtype=torch.int32, device=dev),
            sub=torch.zeros(capacity, dtype=torch.int32, device=dev),
            state=torch.zeros(capacity * 12, dtype=torch.float32, device=dev))
        s = SampleLog(capacity, *[self._log[k].data_ptr() for k in (
            "node", "k", "uraw", "flags", "fail_step", "region", "sub", "state")])
        self._check(lib().kp_set_sample_log(self._ctx, C.byref(s)), "kp_set_sample_log")
        self._log_cap = capacity

    def disable_log(self):
        self._check(lib().kp_set_sample_log(self._ctx, None), "kp_set_sample_log")
        self._log = None

    def read_log(self, n_samples):
        n = min(int(n_samples), self._log_cap)
        self.stream.synchronize()
        out = {}
        for k, v in self._log.items():
            a = v.cpu().numpy()
            if k == "uraw":
                a = a.view(np.uint32).reshape(-1, 4)
            elif k == "state":
                a = a.reshape(-1, 12)[:, : self.d]
            out[k] = a[:n]
        return out

    # ------------------------------------------------------------------
    def attach_mlp(self, mlp, mix=0.5):
        """Learned proposal: mix fraction of samples drawn from the network."""
        self._mlp = mlp
        self._check(lib().kp_attach_mlp(self._ctx, mlp._ctx if mlp is not None else None,
                                        float(mix)), "kp_attach_mlp")

    def set_harvest(self, capacity):
        """Collect (parent features, normalised draw) of every representative
        of a newly reached sub-region into device buffers of 'capacity' rows."""
        import torch
        if capacity is None or capacity <= 0:
            self._check(lib().kp_set_harvest(self._ctx, None, None, 0, None), "kp_set_harvest")
            self._hv = None
            return
        dev = self.device
        self._hv = (torch.zeros((capacity, 32), dtype=torch.float32, device=dev),
                    torch.zeros((capacity, 4), dtype=torch.float32, device=dev),
                    torch.zeros(1, dtype=torch.int32, device=dev), capacity)
        self._check(lib().kp_set_harvest(self._ctx, self._hv[0].data_ptr(), self._hv[1].data_ptr(),
                                         capacity, self._hv[2].data_ptr()), "kp_set_harvest")

    def harvest(self):
        """(features, targets) tensors of the pairs collected so far."""
        self.stream.synchronize()
        n = min(int(self._hv[2].item()), self._hv[3])
        return self._hv[0][:n], self._hv[1][:n]

    def harvest_reset(self):
        self._hv[2].zero_()

    # ------------------------------------------------------------------
    def set_wait_limit(self, ns):
        self._check(lib().kp_set_wait_limit(self._ctx, int(ns)), "kp_set_wait_limit")

    def set_grid_limit(self, max_blocks):
        """Caps the loop launch at max_blocks blocks (0: the resident maximum)."""
        self._check(lib().kp_set_grid_limit(self._ctx, int(max_blocks)), "kp_set_grid_limit")

    def set_extract_ids(self, max_ids):
        """Caps the chain ids the trajectory extraction keeps in shared
        memory (0: the room there); longer chains take the one-thread path."""
        self._check(lib().kp_set_extract_ids(self._ctx, int(max_ids)), "kp_set_extract_ids")

    def selftest_bounds(self):
        return lib().kp_selftest_bounds(self._ctx)

    def selftest_wait_timeout(self):
        return lib().kp_selftest_wait_timeout(self._ctx)

    def last_error(self):
        m = lib().kp_last_error(self._ctx)
        return m.decode() if m else ""
