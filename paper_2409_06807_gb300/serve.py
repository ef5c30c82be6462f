"""Batched planning and serving: thin binding of the kp_server_* entry
points, a real-time arrival driver (continuous batching) and the
autotuner of team size and branching factor.

A server runs one persistent launch whose grid is split into teams of
blocks; each team plans one query at a time and takes the next as soon as
it finishes, so queries that arrive while others run are admitted as soon
as a descriptor slot and device memory for their arena are free.
"""
from __future__ import annotations

import ctypes as C
import time

import numpy as np

from .planner import (OK, NO_SOLUTION, STATUS_NAMES, Budget, KpError, Obstacles, Traj,
                      goal_struct, lib, structs)
from .workloads import STATE_DIM, CONTROL_DIM


class ServerConfig(C.Structure):
    _fields_ = [("team_blocks", C.c_int32), ("max_slots", C.c_int32), ("idle_ms", C.c_double)]


class Done(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int32), ("n_edges", C.c_int32),
                ("iterations", C.c_int32), ("n_nodes", C.c_int32), ("samples", C.c_int64),
                ("device_ms", C.c_double), ("latency_ms", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("teams", C.c_int32), ("team_blocks", C.c_int32), ("pending", C.c_int32),
                ("resident", C.c_int32), ("submitted", C.c_int64), ("completed", C.c_int64),
                ("pool_free", C.c_size_t), ("device_error", C.c_int32), ("running", C.c_int32)]


class Server:
    """A planning server over a device pool (torch uint8 tensor)."""

    def __init__(self, pool_bytes=8 << 30, team_blocks=16, max_slots=512, idle_ms=200.0,
                 device=None, stream=None):
        import torch
        L = lib()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        self.pool = torch.empty(int(pool_bytes), dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        cfg = ServerConfig(int(team_blocks), int(max_slots), float(idle_ms))
        self._ctx = C.c_void_p()
        st = L.kp_server_create(C.byref(cfg), C.c_void_p(self.pool.data_ptr()), int(pool_bytes),
                                C.c_void_p(self.stream.cuda_stream), C.byref(self._ctx))
        if st != OK:
            raise KpError(st, "kp_server_create failed")
        self._buf = (Done * 1024)()
        self.workloads = {}

    def close(self):
        if getattr(self, "_ctx", None):
            lib().kp_server_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, w, max_iters=400, max_ms=0.0) -> int:
        s, ws, p = structs(w)
        boxes = np.ascontiguousarray(np.asarray(w.boxes, np.float32).reshape(-1, 6))
        obs = Obstacles(boxes.ctypes.data_as(C.POINTER(C.c_float)) if len(boxes) else None,
                        len(boxes))
        x = np.ascontiguousarray(w.x_init, np.float32)
        g = goal_struct(w)
        b = Budget(int(max_iters), float(max_ms))
        qid = C.c_int64()
        st = lib().kp_server_submit(self._ctx, C.byref(s), C.byref(ws), C.byref(obs), C.byref(p),
                                    x.ctypes.data_as(C.POINTER(C.c_float)), C.byref(g),
                                    C.byref(b), C.byref(qid))
        if st != OK:
            raise KpError(st, "kp_server_submit failed")
        self.workloads[qid.value] = w
        return qid.value

    def poll(self):
        n = C.c_int32()
        st = lib().kp_server_poll(self._ctx, C.cast(self._buf, C.c_void_p), len(self._buf),
                                  C.byref(n))
        if st != OK:
            raise KpError(st, "kp_server_poll failed")
        return [{f: getattr(self._buf[i], f) for f, _ in Done._fields_} for i in range(n.value)]

    def result(self, qid, capacity=4096):
        w = self.workloads.pop(qid)
        states = np.zeros((capacity, 12), np.float32)
        ctrls = np.zeros((capacity, 4), np.float32)
        steps = np.zeros(capacity, np.int32)
        t = Traj(capacity, 0, states.ctypes.data_as(C.POINTER(C.c_float)),
                 ctrls.ctypes.data_as(C.POINTER(C.c_float)),
                 steps.ctypes.data_as(C.POINTER(C.c_int32)))
        st = lib().kp_server_result(self._ctx, qid, C.byref(t))
        n = t.n_edges if st == OK else 0
        d, m = STATE_DIM[w.system], CONTROL_DIM[w.system]
        return st, dict(states=states[:n, :d], ctrls=ctrls[:n, :m], steps=steps[:n])

    def stats(self):
        s = Stats()
        lib().kp_server_stats_get(self._ctx, C.byref(s))
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def drain(self, timeout_s=120.0, sleep_s=2e-4):
        """Poll until every submitted query has completed."""
        done = []
        t0 = time.perf_counter()
        while True:
            done += self.poll()
            st = self.stats()
            if st["completed"] >= st["submitted"] and st["pending"] == 0 and st["resident"] == 0:
                done += self.poll()
                return done
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError(f"server did not drain: {st}")
            time.sleep(sleep_s)


def run_arrivals(server, arrivals, max_iters=400, timeout_s=300.0):
    """Real-time driver: submits each (t_arrival, workload) at its arrival
    time (relative to the start) and polls completions meanwhile.  Returns
    per-query records with latency measured from arrival to completion."""
    t0 = time.perf_counter()
    ids = {}
    kinds = {}
    recs = []
    i = 0
    while i < len(arrivals) or len(recs) < len(arrivals):
        now = time.perf_counter() - t0
        while i < len(arrivals) and arrivals[i][0] <= now:
            qid = server.submit(arrivals[i][1], max_iters=max_iters)
            ids[qid] = arrivals[i][0]
            kinds[qid] = (arrivals[i][1].system, arrivals[i][1].t_e, len(arrivals[i][1].boxes))
            i += 1
        for d in server.poll():
            t_done = time.perf_counter() - t0
            d["arrival_s"] = ids[d["id"]]
            d["system"], d["t_e"], d["boxes"] = kinds[d["id"]]
            d["done_s"] = t_done
            d["latency_ms"] = 1e3 * (t_done - ids[d["id"]])
            recs.append(d)
        if time.perf_counter() - t0 > timeout_s:
            raise TimeoutError("serving run did not finish")
        if i < len(arrivals):
            nxt = arrivals[i][0] - (time.perf_counter() - t0)
            if nxt > 2e-4:
                time.sleep(min(nxt, 1e-3))
    return recs


def summarize(recs, wall_s):
    lat = np.array([r["latency_ms"] for r in recs])
    ok = np.array([r["status"] == OK for r in recs])
    return dict(queries=len(recs), success=float(ok.mean()) if len(ok) else 0.0,
                p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                queries_per_s=len(recs) / wall_s,
                samples_per_s=float(sum(r["samples"] for r in recs)) / wall_s,
                status={STATUS_NAMES.get(k, k): int(v) for k, v in
                        zip(*np.unique([r["status"] for r in recs], return_counts=True))})


def summarize_by_system(recs):
    """Per system: queries, success rate, latency p50/p99 and, for the
    queries that ended without a solution, their count and the node caps
    they had (a cap below what the system needs fails by construction)."""
    out = {}
    for sysid in sorted({r["system"] for r in recs}):
        rs = [r for r in recs if r["system"] == sysid]
        lat = np.array([r["latency_ms"] for r in rs])
        fail = [r for r in rs if r["status"] != OK]
        out[str(sysid)] = dict(
            queries=len(rs), success=float(np.mean([r["status"] == OK for r in rs])),
            p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
            failures=len(fail),
            failed_t_e_median=float(np.median([r["t_e"] for r in fail])) if fail else None,
            solved_t_e_median=float(np.median([r["t_e"] for r in rs if r["status"] == OK]))
            if len(fail) < len(rs) else None)
    return out


def autotune(sample_queries, team_candidates=(8, 16, 32, 64), lambda_candidates=(32, 64, 128),
             pool_bytes=8 << 30, max_iters=400):
    """Project-written autotuner.  (1) Branching factor: for each system in
    the sample, the lambda_max that solves its queries in the least device
    time per query on a whole-grid team (a property of the query class, so
    a query's lambda never depends on what runs beside it).  (2) Team size:
    the number of blocks per team that gives the highest query throughput
    on the whole sample with those lambdas.  Returns (team_blocks,
    {system: lambda_max}, measurements)."""
    systems = sorted({w.system for w in sample_queries})
    lam = {}
    meas = {"lambda": {}, "team": {}}
    for sysid in systems:
        qs = [w for w in sample_queries if w.system == sysid][:4]
        best = None
        for lm in lambda_candidates:
            srv = Server(pool_bytes, team_blocks=152, max_slots=8)
            t0 = time.perf_counter()
            for w in qs:
                srv.submit(w.with_(lambda_max=lm), max_iters=max_iters)
            done = srv.drain()
            dt = time.perf_counter() - t0
            srv.close()
            score = dt / max(1, sum(d["status"] == OK for d in done))
            meas["lambda"][f"{sysid}:{lm}"] = score
            if best is None or score < best[0]:
                best = (score, lm)
        lam[sysid] = best[1]
    best = None
    for tb in team_candidates:
        srv = Server(pool_bytes, team_blocks=tb, max_slots=256)
        t0 = time.perf_counter()
        for w in sample_queries:
            srv.submit(w.with_(lambda_max=lam[w.system]), max_iters=max_iters)
        srv.drain()
        qps = len(sample_queries) / (time.perf_counter() - t0)
        srv.close()
        meas["team"][tb] = qps
        if best is None or qps > best[0]:
            best = (qps, tb)
    return best[1], lam, meas
