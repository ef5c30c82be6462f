"""Seeded synthetic planning workloads (inputs only).

This module builds the inputs that both the CUDA planner and the CPU oracle
consume: system limits, decomposition grids, planner constants, obstacle
layouts, start states and goal balls.  It holds none of the planner's
arithmetic: no propagation, validity check, binning or estimate.  Every real
value is a float32, so both implementations start from identical numbers.

The paper's benchmark environments (Forest and Building from Ichter et al.
2017, and a Narrow Passage; Sec. VI, Fig. 3) are not available here, so
seeded generators of the same kind stand in for them:

* ``c1``  6D double integrator among 16 random boxes (small case).
* ``c2``  6D Dubins airplane in a forest of 200 vertical boxes.
* ``c3``  12D quadrotor in a building of three walls with one small gap each.
* ``tiny``  hand-sized cases for brute-force tests.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

DI, DUBINS, QUAD = 0, 1, 2
STATE_DIM = {DI: 6, DUBINS: 6, QUAD: 12}
CONTROL_DIM = {DI: 3, DUBINS: 3, QUAD: 4}
INF = np.float32(np.inf)


def _f32(values, n=None, fill=0.0):
    a = np.asarray(values, dtype=np.float32).ravel()
    if n is not None:
        out = np.full(n, fill, dtype=np.float32)
        out[: a.size] = a
        a = out
    return a


@dataclass
class Workload:
    """One planning query: system, decomposition, constants, obstacles."""
    name: str
    system: int
    dt: np.float32
    k_min: int
    k_max: int
    x_lo: np.ndarray          # (12,) float32, +-inf for an unbounded entry
    x_hi: np.ndarray
    u_lo: np.ndarray          # (4,) float32
    u_hi: np.ndarray
    phys: np.ndarray          # (16,) float32
    ws_lo: np.ndarray         # (3,) float32 workspace box
    ws_hi: np.ndarray
    grid: tuple               # region cells per position axis
    speed_bins: int
    speed_hi: np.float32
    sub: tuple                # sub-region cells per region axis
    t_e: int
    lambda_max: int
    delta: float
    eps: float
    seed: int
    boxes: np.ndarray         # (n, 6) float32: lo xyz, hi xyz
    x_init: np.ndarray        # (d,) float32
    goal_c: np.ndarray        # (3,) float32
    goal_r: np.float32
    extra: dict = field(default_factory=dict)
    # cells over state dimension d >= 3 in the region index (0: position
    # grid only); an unbounded dimension (an angle) is wrapped to [-pi, pi)
    state_grid: tuple = (0,) * 12
    # regions are the leaves of a kd-tree split on obstacle faces (a
    # free-space-obeying decomposition); grid, speed bins and state grid
    # are then unused, sub is the sub-grid inside each leaf
    fso: bool = False

    @property
    def d(self) -> int:
        return STATE_DIM[self.system]

    @property
    def n_ctrl(self) -> int:
        return CONTROL_DIM[self.system]

    @property
    def n_regions(self) -> int:
        return int(np.prod(self.grid)) * max(1, self.speed_bins)

    @property
    def n_sub_per(self) -> int:
        return int(np.prod(self.sub))

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


# ---------------------------------------------------------------------------
# systems
# ---------------------------------------------------------------------------

def _di_limits():
    x_lo = _f32([0, 0, 0, -0.3, -0.3, -0.3], 12)
    x_hi = _f32([1, 1, 1, 0.3, 0.3, 0.3], 12)
    return dict(system=DI, dt=np.float32(0.1), k_min=1, k_max=10,
                x_lo=x_lo, x_hi=x_hi,
                u_lo=_f32([-0.5] * 3, 4), u_hi=_f32([0.5] * 3, 4),
                phys=_f32([], 16))


def _dubins_limits():
    th = math.pi / 6
    x_lo = _f32([0, 0, 0, -np.inf, -th, 0.05], 12)
    x_hi = _f32([1, 1, 1, np.inf, th, 0.2], 12)
    return dict(system=DUBINS, dt=np.float32(0.05), k_min=1, k_max=20,
                x_lo=x_lo, x_hi=x_hi,
                u_lo=_f32([-1.0, -0.5, -0.1], 4), u_hi=_f32([1.0, 0.5, 0.1], 4),
                phys=_f32([], 16))


QUAD_PHYS = dict(m=1.0, g=1.0, l=0.05, c=0.01, Ixx=0.01, Iyy=0.01, Izz=0.02)


def _quad_limits():
    a = math.pi / 4
    x_lo = _f32([0, 0, 0, -a, -a, -np.inf, -0.5, -0.5, -0.5, -2, -2, -2], 12)
    x_hi = _f32([1, 1, 1, a, a, np.inf, 0.5, 0.5, 0.5, 2, 2, 2], 12)
    p = QUAD_PHYS
    phys = _f32([p["m"], p["g"], p["l"], p["c"], p["Ixx"], p["Iyy"], p["Izz"]], 16)
    return dict(system=QUAD, dt=np.float32(0.02), k_min=1, k_max=50,
                x_lo=x_lo, x_hi=x_hi,
                u_lo=_f32([0.0] * 4, 4), u_hi=_f32([0.5] * 4, 4), phys=phys)


def _unit_ws():
    return dict(ws_lo=_f32([0, 0, 0]), ws_hi=_f32([1, 1, 1]))


# ---------------------------------------------------------------------------
# obstacle generators
# ---------------------------------------------------------------------------

def _box_hits_ball(box, c, r):
    lo, hi = box[:3].astype(np.float64), box[3:].astype(np.float64)
    q = np.clip(np.asarray(c, np.float64), lo, hi)
    return float(np.sum((q - c) ** 2)) <= r * r


def random_boxes(seed: int, n: int = 16, side=(0.05, 0.15), keep_clear=()):
    """n axis-aligned boxes in the unit cube; sides U[side], centres U[0,1]^3,
    clipped to the cube; a box that meets a keep-clear ball is redrawn."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    while len(out) < n:
        c = rng.uniform(0.0, 1.0, 3)
        s = rng.uniform(side[0], side[1], 3)
        box = np.concatenate([np.clip(c - s / 2, 0, 1), np.clip(c + s / 2, 0, 1)])
        box = box.astype(np.float32)
        if any(_box_hits_ball(box, cc, rr) for cc, rr in keep_clear):
            continue
        out.append(box)
    return np.stack(out).astype(np.float32)


def forest_boxes(seed: int, n: int = 200, width=(0.02, 0.04), keep_clear=()):
    """n vertical 'trunks' spanning z in [0, 1]; x/y widths U[width], centres
    U[0,1]^2; a trunk that meets a keep-clear ball is redrawn."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    while len(out) < n:
        c = rng.uniform(0.0, 1.0, 2)
        w = rng.uniform(width[0], width[1], 2)
        lo = np.clip(c - w / 2, 0, 1)
        hi = np.clip(c + w / 2, 0, 1)
        box = np.array([lo[0], lo[1], 0.0, hi[0], hi[1], 1.0], dtype=np.float32)
        if any(_box_hits_ball(box, cc, rr) for cc, rr in keep_clear):
            continue
        out.append(box)
    return np.stack(out).astype(np.float32)


def building_boxes(seed: int, walls=(0.25, 0.5, 0.75), thickness=0.02,
                   tiles=20, gap=0.06):
    """Walls normal to x.  Each wall tiles the y-z square with tiles x tiles
    boxes whose gap row and gap column are 'gap' wide (the others share the
    rest equally); the gap tile is left out, leaving one gap x gap hole at a
    seeded place.  One zero-volume box outside the workspace pads each wall
    to tiles^2 boxes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for wx in walls:
        gy, gz = rng.integers(1, tiles - 1, size=2)
        rest = (1.0 - gap) / (tiles - 1)

        def edges(g):
            w = np.full(tiles, rest)
            w[g] = gap
            return np.concatenate([[0.0], np.cumsum(w)])

        ey, ez = edges(gy), edges(gz)
        ey[-1] = ez[-1] = 1.0
        for iy in range(tiles):
            for iz in range(tiles):
                if iy == gy and iz == gz:
                    continue
                out.append([wx - thickness / 2, ey[iy], ez[iz],
                            wx + thickness / 2, ey[iy + 1], ez[iz + 1]])
        out.append([2.0, 2.0, 2.0, 2.0, 2.0, 2.0])  # padding, outside W
    return np.asarray(out, dtype=np.float32)


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def c1(seed: int = 0, **kw) -> Workload:
    """6D double integrator, 16 random boxes, 8^3 regions x 4^3 sub-regions,
    lambda_max 32, t_e 65,536, goal ball r = 0.05."""
    start, goal, r = (0.1, 0.1, 0.1), (0.9, 0.9, 0.9), 0.05
    boxes = random_boxes(seed, 16, keep_clear=[(start, 0.0), (goal, r)])
    w = Workload(name="c1_double_integrator", **_di_limits(), **_unit_ws(),
                 grid=(8, 8, 8), speed_bins=1, speed_hi=np.float32(1.0),
                 sub=(4, 4, 4), t_e=65536, lambda_max=32, delta=1.0, eps=0.01,
                 seed=seed, boxes=boxes,
                 x_init=_f32([*start, 0, 0, 0]),
                 goal_c=_f32(goal), goal_r=np.float32(r))
    return w.with_(**kw) if kw else w


def c2(seed: int = 0, **kw) -> Workload:
    """6D Dubins airplane in a 200-trunk forest, 16^3 regions x 4^3
    sub-regions, lambda_max 64, t_e 1,048,576, start and goal at opposite
    corners."""
    start, goal, r = (0.05, 0.05, 0.5), (0.95, 0.95, 0.5), 0.05
    boxes = forest_boxes(seed, 200, keep_clear=[(start, 0.03), (goal, r)])
    w = Workload(name="c2_dubins_forest", **_dubins_limits(), **_unit_ws(),
                 grid=(16, 16, 16), speed_bins=1, speed_hi=np.float32(1.0),
                 sub=(4, 4, 4), t_e=1 << 20, lambda_max=64, delta=1.0,
                 eps=0.01, seed=seed, boxes=boxes,
                 x_init=_f32([*start, math.pi / 4, 0.0, 0.1]),
                 goal_c=_f32(goal), goal_r=np.float32(r))
    return w.with_(**kw) if kw else w


def c3(seed: int = 0, **kw) -> Workload:
    """12D quadrotor in a three-wall building (1,200 boxes), 16^3 position
    regions x 4 speed bins, 4^3 sub-regions, lambda_max 128, t_e 4,194,304,
    start at hover."""
    boxes = building_boxes(seed)
    x0 = np.zeros(12, dtype=np.float32)
    x0[:3] = (0.1, 0.5, 0.5)
    w = Workload(name="c3_quadrotor_building", **_quad_limits(), **_unit_ws(),
                 grid=(16, 16, 16), speed_bins=4, speed_hi=np.float32(0.5),
                 sub=(4, 4, 4), t_e=1 << 22, lambda_max=128, delta=1.0,
                 eps=0.01, seed=seed, boxes=boxes, x_init=x0,
                 goal_c=_f32([0.9, 0.5, 0.5]), goal_r=np.float32(0.05))
    return w.with_(**kw) if kw else w


def tiny(system: int = DI, seed: int = 0, n_boxes: int = 2, **kw) -> Workload:
    """Hand-sized case: 2^3 regions x 2^3 sub-regions, small lambda and t_e."""
    lim = {DI: _di_limits, DUBINS: _dubins_limits, QUAD: _quad_limits}[system]()
    d = STATE_DIM[system]
    x0 = np.zeros(d, dtype=np.float32)
    x0[:3] = (0.2, 0.2, 0.5)
    if system == DUBINS:
        x0[3:6] = (math.pi / 4, 0.0, 0.1)
    boxes = random_boxes(seed, n_boxes, side=(0.1, 0.2),
                         keep_clear=[(tuple(x0[:3]), 0.05), ((0.8, 0.8, 0.5), 0.1)]) \
        if n_boxes else np.zeros((0, 6), np.float32)
    w = Workload(name=f"tiny_{system}", **lim, **_unit_ws(), grid=(2, 2, 2),
                 speed_bins=1, speed_hi=np.float32(1.0), sub=(2, 2, 2),
                 t_e=512, lambda_max=4, delta=1.0, eps=0.01, seed=seed,
                 boxes=boxes, x_init=x0, goal_c=_f32([0.8, 0.8, 0.5]),
                 goal_r=np.float32(0.1))
    return w.with_(**kw) if kw else w


def serving_mix(n: int = 512, rate_hz: float = 2000.0, seed: int = 0, t_e_range=(16384, 1 << 20),
                box_range=(10, 1000)):
    """Arrival process of mixed queries: Poisson arrivals at rate_hz; system
    uniform over the three; obstacle count and node cap log-uniform in the
    given ranges; each layout from its system's generator (random boxes,
    forest or building walls, with the count drawn).  Returns a list of
    (arrival time in s, Workload)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n))
    out = []
    for i in range(n):
        system = int(rng.integers(0, 3))
        nb = int(round(np.exp(rng.uniform(np.log(box_range[0]), np.log(box_range[1])))))
        t_e = int(round(np.exp(rng.uniform(np.log(t_e_range[0]), np.log(t_e_range[1])))))
        s = int(rng.integers(0, 2 ** 31))
        if system == DI:
            w = c1(s).with_(t_e=t_e)
            w = w.with_(boxes=random_boxes(s, nb, keep_clear=[(tuple(w.x_init[:3]), 0.0),
                                                              (tuple(w.goal_c), float(w.goal_r))]))
        elif system == DUBINS:
            w = c2(s).with_(t_e=t_e)
            w = w.with_(boxes=forest_boxes(s, nb, keep_clear=[(tuple(w.x_init[:3]), 0.03),
                                                              (tuple(w.goal_c), float(w.goal_r))]))
        else:
            w = c3(s).with_(t_e=t_e)
            per_wall = max(1, nb // 3)
            walls = building_boxes(s)
            w = w.with_(boxes=np.concatenate([walls[k * 400:k * 400 + per_wall] for k in range(3)]))
        out.append((float(t[i]), w.with_(name=f"{w.name}_q{i}")))
    return out


BY_NAME = {"c1": c1, "c2": c2, "c3": c3}
