"""ctypes binding of the FP64 CPU oracle (``libkpo.so``).

TEST INFRASTRUCTURE ONLY: used by the test suite, the package smoke check
and the benchmark's CPU-baseline leg to check and time the CUDA planner.  It
never imports the CUDA package; callers hand it a workload object (any object
with the attributes of ``paper_2409_06807_gb300.workloads.Workload``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import build_oracle

RUNNING, SOLVED, FULL, ERR = 0, 1, 2, -1

_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")


class Config(C.Structure):
    _fields_ = [
        ("system", C.c_int32), ("dt", C.c_double),
        ("k_min", C.c_int32), ("k_max", C.c_int32),
        ("x_lo", C.c_double * 12), ("x_hi", C.c_double * 12),
        ("u_lo", C.c_double * 4), ("u_hi", C.c_double * 4),
        ("phys", C.c_double * 16),
        ("ws_lo", C.c_double * 3), ("ws_hi", C.c_double * 3),
        ("grid", C.c_int32 * 3), ("speed_bins", C.c_int32),
        ("speed_hi", C.c_double), ("sub", C.c_int32 * 3), ("fso", C.c_int32),
        ("state_grid", C.c_int32 * 12),
        ("t_e", C.c_int32), ("lambda_max", C.c_int32),
        ("delta", C.c_double), ("eps", C.c_double),
        ("seed", C.c_uint64),
        ("goal_c", C.c_double * 3), ("goal_r", C.c_double),
    ]


class Records(C.Structure):
    _fields_ = [
        ("capacity", C.c_int32),
        ("node", C.POINTER(C.c_int32)), ("k", C.POINTER(C.c_int32)),
        ("uraw", C.POINTER(C.c_uint32)), ("flags", C.POINTER(C.c_uint8)),
        ("fail_step", C.POINTER(C.c_int32)), ("region", C.POINTER(C.c_int32)),
        ("sub", C.POINTER(C.c_int32)), ("state", C.POINTER(C.c_double)),
        ("m_valid", C.POINTER(C.c_double)), ("m_bin", C.POINTER(C.c_double)),
        ("m_goal", C.POINTER(C.c_double)),
    ]


class Work(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("samples", "steps", "hulls", "box_scan", "box_grid",
                                           "ops")]


class IterStats(C.Structure):
    _fields_ = [(n, C.c_int32) for n in (
        "iteration", "n_ve", "lambda_", "n_samples", "n_valid", "n_accepted",
        "n_nodes", "goal_node")]

    def as_dict(self):
        return {n if n != "lambda_" else "lambda": getattr(self, n)
                for n, _ in self._fields_}


_lib = None


def lib():
    global _lib
    if _lib is None:
        # KPO_LIB names another build of these sources (the mutation check
        # of the tests loads copies with a planted mistake this way)
        L = C.CDLL(os.environ.get("KPO_LIB") or build_oracle())
        vp = C.c_void_p
        L.kpo_create.restype = vp
        L.kpo_create.argtypes = [C.POINTER(Config), _f32p, C.c_int32]
        L.kpo_destroy.argtypes = [vp]
        for name in ("kpo_state_dim", "kpo_control_dim", "kpo_num_regions",
                     "kpo_num_subregions", "kpo_status", "kpo_goal_node",
                     "kpo_num_nodes", "kpo_iteration"):
            getattr(L, name).restype = C.c_int32
            getattr(L, name).argtypes = [vp]
        L.kpo_reset.restype = C.c_int32
        L.kpo_reset.argtypes = [vp, _f32p]
        L.kpo_iterate.restype = C.c_int32
        L.kpo_iterate.argtypes = [vp, C.POINTER(Records), C.POINTER(IterStats)]
        L.kpo_run.restype = C.c_int32
        L.kpo_run.argtypes = [vp, C.c_int32, C.POINTER(C.c_int32)]
        L.kpo_export.argtypes = [vp, _f64p, _i32p, _f64p, _i32p, _i32p, _i32p,
                                 _u8p, _u32p, _u32p, _u32p, _u8p, _u64p, _u8p]
        L.kpo_import.restype = C.c_int32
        L.kpo_import.argtypes = [vp, C.c_int32, C.c_int32, _f32p, _i32p, _f32p,
                                 _i32p, _i32p, _i32p, _u8p, _u32p, _u32p,
                                 _u64p, _u8p]
        L.kpo_estimates.argtypes = [vp, _f64p, _f64p, C.POINTER(C.c_double)]
        L.kpo_path.restype = C.c_int32
        L.kpo_path.argtypes = [vp, _i32p, C.c_int32]
        L.kpo_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.kpo_philox4x32_10_n.argtypes = [_u32p, _u32p, _u32p, C.c_int64]
        L.kpo_region_volumes.argtypes = [vp, _f64p]
        L.kpo_set_work_grid.argtypes = [vp, _i32p]
        L.kpo_get_work.argtypes = [vp, C.POINTER(Work)]
        L.kpo_clear_work.argtypes = [vp]
        L.kpo_work_clearance.restype = C.c_int32
        L.kpo_work_clearance.argtypes = [vp, _i32p]
        for name in ("kpo_work_ops_sample", "kpo_work_ops_step"):
            getattr(L, name).restype = C.c_uint64
            getattr(L, name).argtypes = [vp]
        for name in ("kpo_work_ops_hull", "kpo_work_ops_box"):
            getattr(L, name).restype = C.c_uint64
            getattr(L, name).argtypes = []
        L.kpo_step.argtypes = [C.POINTER(Config), _f64p, _f64p, C.c_double, _f64p]
        L.kpo_propagate.argtypes = [C.POINTER(Config), _f64p, _f64p, C.c_int32, _f64p]
        L.kpo_step_valid.restype = C.c_int32
        L.kpo_step_valid.argtypes = [vp, _f64p, _f64p, C.POINTER(C.c_double)]
        L.kpo_bin.argtypes = [vp, _f64p, C.POINTER(C.c_int32),
                              C.POINTER(C.c_int32), C.POINTER(C.c_double)]
        L.kpo_eq345.argtypes = [C.c_int32, _u32p, _u32p, _u32p, _u8p, C.c_double,
                                C.c_double, C.c_double, _f64p, _f64p, _u64p,
                                C.POINTER(C.c_double)]
        L.kpo_lambda.restype = C.c_int32
        L.kpo_lambda.argtypes = [C.c_int32] * 4
        L.kpo_mlp_num_params.restype = C.c_int32
        L.kpo_mlp_num_params.argtypes = []
        L.kpo_mlp_forward.argtypes = [_f64p, _f64p, C.c_int32, _f64p]
        L.kpo_mlp_loss_grad.restype = C.c_double
        L.kpo_mlp_loss_grad.argtypes = [_f64p, _f64p, _f64p, C.c_int32, C.c_void_p]
        L.kpo_adam.argtypes = [_f64p, _f64p, _f64p, _f64p, C.c_int32, C.c_double, C.c_double,
                               C.c_double, C.c_double, C.c_int32]
        L.kpo_features.argtypes = [vp, C.c_int32, _f64p]
        L.kpo_set_mlp.restype = C.c_int32
        L.kpo_set_mlp.argtypes = [vp, C.c_void_p, C.c_double]
        L.kpo_set_harvest.restype = C.c_int32
        L.kpo_set_harvest.argtypes = [vp, C.c_void_p, C.c_void_p, C.c_int32]
        L.kpo_harvest_count.restype = C.c_int32
        L.kpo_harvest_count.argtypes = [vp]
        L.kpo_box_muller.argtypes = [_u32p, _f64p]
        L.kpo_fso_leaves.restype = C.c_int32
        L.kpo_fso_leaves.argtypes = [vp, _f64p, _f64p, C.c_int32]
        L.kpo_eq345_vol.argtypes = [C.c_int32, _u32p, _u32p, _u32p, _u8p, _f64p,
                                    C.c_double, C.c_double, _f64p, _f64p, _u64p,
                                    C.POINTER(C.c_double)]
        L.kpo_dense_check.restype = C.c_double
        L.kpo_dense_check.argtypes = [vp, _f64p, _f64p, C.c_int32, C.c_int32, _f64p]
        _lib = L
    return _lib


def make_config(w) -> Config:
    c = Config()
    c.system = int(w.system)
    c.dt = float(np.float32(w.dt))
    c.k_min, c.k_max = int(w.k_min), int(w.k_max)
    for i in range(12):
        c.x_lo[i] = float(w.x_lo[i])
        c.x_hi[i] = float(w.x_hi[i])
    for i in range(4):
        c.u_lo[i] = float(w.u_lo[i])
        c.u_hi[i] = float(w.u_hi[i])
    for i in range(16):
        c.phys[i] = float(w.phys[i])
    for i in range(3):
        c.ws_lo[i] = float(w.ws_lo[i])
        c.ws_hi[i] = float(w.ws_hi[i])
        c.grid[i] = int(w.grid[i])
        c.sub[i] = int(w.sub[i])
        c.goal_c[i] = float(w.goal_c[i])
    c.speed_bins = int(w.speed_bins)
    for i in range(12):
        c.state_grid[i] = int(w.state_grid[i])
    c.fso = 1 if getattr(w, "fso", False) else 0
    c.speed_hi = float(np.float32(w.speed_hi))
    c.t_e, c.lambda_max = int(w.t_e), int(w.lambda_max)
    c.delta, c.eps = float(w.delta), float(w.eps)
    c.seed = int(w.seed) & 0xFFFFFFFFFFFFFFFF
    c.goal_r = float(np.float32(w.goal_r))
    return c


def philox4x32_10(ctr, key) -> np.ndarray:
    out = np.zeros(4, np.uint32)
    lib().kpo_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def philox4x32_10_n(ctrs, key) -> np.ndarray:
    """Philox blocks of many counters ([n][4]) under one key ([n][4] words)."""
    c = np.ascontiguousarray(ctrs, np.uint32).reshape(-1, 4)
    out = np.zeros_like(c)
    lib().kpo_philox4x32_10_n(c.reshape(-1), np.asarray(key, np.uint32), out.reshape(-1),
                              len(c))
    return out


def eq345(n_valid, n_invalid, cov, avail, vol, delta, eps):
    n = len(n_valid)
    score = np.zeros(n)
    p = np.zeros(n)
    thr = np.zeros(n, np.uint64)
    s = C.c_double()
    lib().kpo_eq345(n, np.ascontiguousarray(n_valid, np.uint32),
                    np.ascontiguousarray(n_invalid, np.uint32),
                    np.ascontiguousarray(cov, np.uint32),
                    np.ascontiguousarray(avail, np.uint8), vol, delta, eps,
                    score, p, thr, C.byref(s))
    return score, p, thr, s.value


def eq345_vol(n_valid, n_invalid, cov, avail, vol_r, delta, eps):
    """Eq. 3-5 with a volume per region."""
    n = len(n_valid)
    score = np.zeros(n)
    p = np.zeros(n)
    thr = np.zeros(n, np.uint64)
    s = C.c_double()
    lib().kpo_eq345_vol(n, np.ascontiguousarray(n_valid, np.uint32),
                        np.ascontiguousarray(n_invalid, np.uint32),
                        np.ascontiguousarray(cov, np.uint32),
                        np.ascontiguousarray(avail, np.uint8),
                        np.ascontiguousarray(vol_r, np.float64), delta, eps,
                        score, p, thr, C.byref(s))
    return score, p, thr, s.value


MLP_IN, MLP_H, MLP_OUT = 32, 256, 8


def mlp_num_params() -> int:
    return lib().kpo_mlp_num_params()


def mlp_forward(params, x) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float64).reshape(-1, MLP_IN)
    out = np.zeros((len(x), MLP_OUT))
    lib().kpo_mlp_forward(np.ascontiguousarray(params, np.float64), x, len(x), out.reshape(-1))
    return out


def mlp_loss_grad(params, x, t, grad=True):
    x = np.ascontiguousarray(x, np.float64).reshape(-1, MLP_IN)
    t = np.ascontiguousarray(t, np.float64).reshape(-1, 4)
    g = np.zeros(mlp_num_params()) if grad else None
    loss = lib().kpo_mlp_loss_grad(np.ascontiguousarray(params, np.float64), x.reshape(-1),
                                   t.reshape(-1), len(x),
                                   g.ctypes.data if grad else None)
    return loss, g


def adam(p, g, m, v, lr, t, beta1=0.9, beta2=0.999, eps=1e-8):
    lib().kpo_adam(p, np.ascontiguousarray(g, np.float64), m, v, len(p), lr, beta1, beta2,
                   eps, t)


def box_muller(words) -> np.ndarray:
    z = np.zeros(4)
    lib().kpo_box_muller(np.ascontiguousarray(words, np.uint32), z)
    return z


def mlp_split(p):
    """Views (W1, b1, W2, b2, W3, b3) of a flat parameter vector."""
    sizes = [(MLP_H, MLP_IN), (MLP_H,), (MLP_H, MLP_H), (MLP_H,), (MLP_OUT, MLP_H), (MLP_OUT,)]
    out, o = [], 0
    for s in sizes:
        n = int(np.prod(s))
        out.append(p[o:o + n].reshape(s))
        o += n
    return out


def lam(t_e, n_tree, n_ve, lambda_max) -> int:
    return lib().kpo_lambda(t_e, n_tree, n_ve, lambda_max)


def step(w, x, u, h=None) -> np.ndarray:
    cfg = make_config(w)
    out = np.zeros(len(x))
    lib().kpo_step(C.byref(cfg), np.asarray(x, np.float64), _pad(u, 4),
                   float(cfg.dt if h is None else h), out)
    return out


def propagate(w, x0, u, k) -> np.ndarray:
    cfg = make_config(w)
    d = len(x0)
    traj = np.zeros((k + 1) * d)
    lib().kpo_propagate(C.byref(cfg), np.asarray(x0, np.float64), _pad(u, 4), k, traj)
    return traj.reshape(k + 1, d)


def _pad(u, n):
    a = np.zeros(n)
    u = np.asarray(u, np.float64).ravel()
    a[: u.size] = u
    return a


class Oracle:
    """One planner instance of the oracle (Algorithm 1 state)."""

    def __init__(self, w):
        self.w = w
        self._cfg = make_config(w)
        boxes = np.ascontiguousarray(np.asarray(w.boxes, np.float32).reshape(-1))
        if boxes.size == 0:
            boxes = np.zeros(6, np.float32)
        L = lib()
        self._h = L.kpo_create(C.byref(self._cfg), boxes, int(len(w.boxes)))
        if not self._h:
            raise ValueError("oracle rejected the configuration")
        self.d = L.kpo_state_dim(self._h)
        self.N = L.kpo_control_dim(self._h)
        self.R = L.kpo_num_regions(self._h)
        self.n_sub = L.kpo_num_subregions(self._h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().kpo_destroy(h)
            self._h = None

    # -- Algorithm 1 ------------------------------------------------------
    def reset(self, x_init=None) -> int:
        x = self.w.x_init if x_init is None else x_init
        return lib().kpo_reset(self._h, np.ascontiguousarray(x, np.float32))

    def iterate(self, records: bool = False, capacity: int | None = None):
        """One loop pass.  Returns (status, stats dict, records dict|None)."""
        st = IterStats()
        rec = None
        arrays = None
        if records:
            cap = capacity or self.w.t_e
            arrays = dict(
                node=np.full(cap, -1, np.int32), k=np.zeros(cap, np.int32),
                uraw=np.zeros(4 * cap, np.uint32), flags=np.zeros(cap, np.uint8),
                fail_step=np.zeros(cap, np.int32), region=np.zeros(cap, np.int32),
                sub=np.zeros(cap, np.int32), state=np.zeros(cap * self.d),
                m_valid=np.zeros(cap), m_bin=np.zeros(cap), m_goal=np.zeros(cap))
            rec = Records()
            rec.capacity = cap
            for name, a in arrays.items():
                ct = np.ctypeslib.as_ctypes_type(a.dtype)
                setattr(rec, name, a.ctypes.data_as(C.POINTER(ct)))
        status = lib().kpo_iterate(self._h, C.byref(rec) if rec else None, C.byref(st))
        out = None
        if records:
            S = st.n_samples
            out = {k: (v[: 4 * S].reshape(S, 4) if k == "uraw" else
                       v[: S * self.d].reshape(S, self.d) if k == "state" else v[:S])
                   for k, v in arrays.items()}
        return status, st.as_dict(), out

    def run(self, max_iters: int):
        done = C.c_int32()
        status = lib().kpo_run(self._h, max_iters, C.byref(done))
        return status, done.value

    @property
    def status(self):
        return lib().kpo_status(self._h)

    @property
    def goal_node(self):
        return lib().kpo_goal_node(self._h)

    @property
    def n_nodes(self):
        return lib().kpo_num_nodes(self._h)

    @property
    def iteration(self):
        return lib().kpo_iteration(self._h)

    # -- state I/O ----------------------------------------------------------
    def export(self) -> dict:
        n = self.n_nodes
        t = dict(
            state=np.zeros((n, self.d)), parent=np.zeros(n, np.int32),
            ctrl=np.zeros((n, self.N)), steps=np.zeros(n, np.int32),
            region=np.zeros(n, np.int32), sub=np.zeros(n, np.int32),
            in_ve=np.zeros(n, np.uint8), n_valid=np.zeros(self.R, np.uint32),
            n_invalid=np.zeros(self.R, np.uint32), cov=np.zeros(self.R, np.uint32),
            avail=np.zeros(self.R, np.uint8), thr=np.zeros(self.R, np.uint64),
            visited=np.zeros(self.n_sub, np.uint8))
        lib().kpo_export(self._h, t["state"].reshape(-1), t["parent"],
                         t["ctrl"].reshape(-1), t["steps"], t["region"], t["sub"],
                         t["in_ve"], t["n_valid"], t["n_invalid"], t["cov"],
                         t["avail"], t["thr"], t["visited"])
        t["iteration"] = self.iteration
        t["n_nodes"] = n
        return t

    def import_(self, t: dict) -> None:
        n = int(t["n_nodes"])
        rc = lib().kpo_import(
            self._h, n, int(t["iteration"]),
            np.ascontiguousarray(t["state"], np.float32).reshape(-1),
            np.ascontiguousarray(t["parent"], np.int32),
            np.ascontiguousarray(t["ctrl"], np.float32).reshape(-1),
            np.ascontiguousarray(t["steps"], np.int32),
            np.ascontiguousarray(t["region"], np.int32),
            np.ascontiguousarray(t["sub"], np.int32),
            np.ascontiguousarray(t["in_ve"], np.uint8),
            np.ascontiguousarray(t["n_valid"], np.uint32),
            np.ascontiguousarray(t["n_invalid"], np.uint32),
            np.ascontiguousarray(t["thr"], np.uint64),
            np.ascontiguousarray(t["visited"], np.uint8))
        if rc != RUNNING:
            raise ValueError("oracle rejected the imported tree")

    def estimates(self):
        score = np.zeros(self.R)
        p = np.zeros(self.R)
        s = C.c_double()
        lib().kpo_estimates(self._h, score, p, C.byref(s))
        return score, p, s.value

    def path(self) -> np.ndarray:
        cap = self.n_nodes
        out = np.zeros(max(cap, 1), np.int32)
        n = lib().kpo_path(self._h, out, cap)
        return out[:n]

    # -- building blocks ---------------------------------------------------
    def step_valid(self, x0, x1):
        m = C.c_double()
        ok = lib().kpo_step_valid(self._h, np.asarray(x0, np.float64),
                                  np.asarray(x1, np.float64), C.byref(m))
        return bool(ok), m.value

    def bin(self, x):
        r, s, m = C.c_int32(), C.c_int32(), C.c_double()
        lib().kpo_bin(self._h, np.asarray(x, np.float64), C.byref(r), C.byref(s),
                      C.byref(m))
        return r.value, s.value, m.value

    def set_work_grid(self, g):
        """Broad-phase grid (cells per position axis) of the pruned box count."""
        lib().kpo_set_work_grid(self._h, np.ascontiguousarray(g, np.int32))

    def work(self) -> dict:
        """Work counted since the last reset or import (see oracle/work.c)."""
        wk = Work()
        lib().kpo_get_work(self._h, C.byref(wk))
        return {n: int(getattr(wk, n)) for n, _ in Work._fields_}

    def work_clearance(self) -> np.ndarray:
        """Cell clearances (sixteenths of a cell) of the work grid."""
        out = np.zeros(4096 * 16, np.int32)
        n = lib().kpo_work_clearance(self._h, out)
        return out[:n]

    def clear_work(self):
        lib().kpo_clear_work(self._h)

    def work_costs(self) -> dict:
        """Lane operations per sample, integrator step, hull and box test."""
        L = lib()
        return {"sample": int(L.kpo_work_ops_sample(self._h)),
                "step": int(L.kpo_work_ops_step(self._h)),
                "hull": int(L.kpo_work_ops_hull()), "box": int(L.kpo_work_ops_box())}

    def region_volumes(self) -> np.ndarray:
        """Volume of every region in Eq. 3 (grid cell or kd-tree leaf)."""
        v = np.zeros(self.R)
        lib().kpo_region_volumes(self._h, v)
        return v

    def fso_leaves(self):
        """Leaf boxes (lo, hi), each (n_leaves, 3), of the free-space-obeying
        decomposition in region order; None for a grid."""
        lo = np.zeros((16384, 3))
        hi = np.zeros((16384, 3))
        n = lib().kpo_fso_leaves(self._h, lo, hi, 16384)
        return (lo[:n], hi[:n]) if n else None

    def features(self, v) -> np.ndarray:
        f = np.zeros(32)
        lib().kpo_features(self._h, int(v), f)
        return f

    def set_mlp(self, params, mix=0.5):
        if params is None:
            self._mlp = None
            lib().kpo_set_mlp(self._h, None, 0.0)
            return
        self._mlp = np.ascontiguousarray(params, np.float32)
        if lib().kpo_set_mlp(self._h, self._mlp.ctypes.data, float(mix)) != 0:
            raise ValueError("learned proposal needs a 6D system")

    def set_harvest(self, capacity):
        self._hv = (np.zeros((capacity, 32)), np.zeros((capacity, 4)))
        lib().kpo_set_harvest(self._h, self._hv[0].ctypes.data, self._hv[1].ctypes.data,
                              int(capacity))

    def harvest(self):
        n = lib().kpo_harvest_count(self._h)
        return self._hv[0][:n].copy(), self._hv[1][:n].copy()

    def dense_check(self, x0, u, k, sub=100):
        x_end = np.zeros(self.d)
        depth = lib().kpo_dense_check(self._h, np.asarray(x0, np.float64),
                                      _pad(u, 4), int(k), int(sub), x_end)
        return depth, x_end
