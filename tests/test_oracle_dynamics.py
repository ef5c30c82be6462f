"""Pins of the oracle's propagation (Sec. II, Eq. 1-2) against closed forms."""
import math

import numpy as np

from paper_2409_06807_gb300 import workloads as W


def test_double_integrator_euler_closed_form(kpo):
    """Explicit Euler with constant a over k steps:
    v_k = v0 + k a h,  p_k = p0 + k v0 h + a h^2 k (k - 1) / 2."""
    w = W.c1(0)
    h = float(np.float32(w.dt))
    rng = np.random.default_rng(1)
    for _ in range(20):
        x0 = rng.uniform(-1, 1, 6)
        a = rng.uniform(-0.5, 0.5, 3)
        k = int(rng.integers(1, 11))
        traj = kpo.propagate(w, x0, a, k)
        for i in range(k + 1):
            v = x0[3:] + i * a * h
            p = x0[:3] + i * x0[3:] * h + a * h * h * i * (i - 1) / 2
            np.testing.assert_allclose(traj[i, 3:], v, atol=1e-12)
            np.testing.assert_allclose(traj[i, :3], p, atol=1e-12)


def test_dubins_straight_line(kpo):
    """Zero turn rates and zero acceleration: straight flight at speed v."""
    w = W.c2(0)
    x0 = np.array([0.2, 0.3, 0.4, 0.7, 0.2, 0.15])
    k = 20
    traj = kpo.propagate(w, x0, [0, 0, 0], k)
    t = k * float(np.float32(w.dt))
    v, psi, th = x0[5], x0[3], x0[4]
    exp = x0[:3] + t * v * np.array([math.cos(psi) * math.cos(th),
                                     math.sin(psi) * math.cos(th), math.sin(th)])
    np.testing.assert_allclose(traj[-1, :3], exp, atol=1e-13)
    np.testing.assert_allclose(traj[-1, 3:], x0[3:], atol=0)


def test_dubins_constant_acceleration(kpo):
    """Level straight flight with constant acceleration: x = v0 t + a t^2/2
    (a quadratic, which RK4 integrates exactly)."""
    w = W.c2(0)
    x0 = np.array([0.1, 0.1, 0.5, 0.0, 0.0, 0.1])
    a = 0.05
    k = 20
    traj = kpo.propagate(w, x0, [0, 0, a], k)
    t = k * float(np.float32(w.dt))
    assert abs(traj[-1, 0] - (0.1 + 0.1 * t + a * t * t / 2)) < 1e-13
    assert abs(traj[-1, 5] - (0.1 + a * t)) < 1e-13


def _helix(x0, omega, t):
    psi0, th, v = x0[3], x0[4], x0[5]
    r = v * math.cos(th) / omega
    psi = psi0 + omega * t
    return np.array([x0[0] + r * (math.sin(psi) - math.sin(psi0)),
                     x0[1] - r * (math.cos(psi) - math.cos(psi0)),
                     x0[2] + v * math.sin(th) * t])


def test_dubins_helix_and_rk4_order(kpo):
    """Constant yaw rate: a helix of radius v cos(theta)/omega.  RK4 error
    falls by ~2^4 each time the step halves."""
    w = W.c2(0)
    x0 = np.array([0.5, 0.5, 0.5, 0.3, 0.1, 0.2])
    omega, t_end = 1.0, 1.0
    errs = []
    for n in (10, 20, 40):
        h = t_end / n
        x = x0.copy()
        for _ in range(n):
            x = kpo.step(w, x, [omega, 0, 0], h)
        errs.append(np.linalg.norm(x[:3] - _helix(x0, omega, t_end)))
    assert errs[0] < 1e-6
    for a, b in zip(errs, errs[1:]):
        assert 12.0 < a / b < 20.0


def test_quadrotor_hover_is_fixed_point(kpo):
    w = W.c3(0)
    x0 = np.zeros(12)
    x0[:3] = (0.3, 0.4, 0.5)
    x0[5] = 0.7  # any yaw
    traj = kpo.propagate(w, x0, [0.25] * 4, 50)
    np.testing.assert_allclose(traj[-1], x0, atol=1e-14)


def test_quadrotor_pure_yaw(kpo):
    """T1 = T3 = a, T2 = T4 = b with a + b = m g / 2: zero net force and
    roll/pitch torque; yaw accelerates at 2 c (a - b) / Izz, so
    psi(t) = psi0 + r0 t + alpha t^2 / 2 (exact under RK4)."""
    w = W.c3(0)
    p = W.QUAD_PHYS
    a, b = 0.3, 0.2
    alpha = 2 * p["c"] * (a - b) / p["Izz"]
    x0 = np.zeros(12)
    x0[:3] = (0.5, 0.5, 0.5)
    x0[11] = 0.2
    k = 50
    traj = kpo.propagate(w, x0, [a, b, a, b], k)
    t = k * float(np.float32(w.dt))
    assert abs(traj[-1, 5] - (0.2 * t + alpha * t * t / 2)) < 1e-12
    assert abs(traj[-1, 11] - (0.2 + alpha * t)) < 1e-12
    np.testing.assert_allclose(traj[-1, :3], x0[:3], atol=1e-14)
    np.testing.assert_allclose(traj[-1, 6:11], 0.0, atol=1e-14)


def test_quadrotor_free_fall_and_climb(kpo):
    """Level attitude, total thrust F: vertical acceleration F/m - g."""
    w = W.c3(0)
    x0 = np.zeros(12)
    x0[:3] = (0.5, 0.5, 0.5)
    for thrust in (0.0, 0.6, 1.8):
        k = 25
        traj = kpo.propagate(w, x0, [thrust / 4] * 4, k)
        t = k * float(np.float32(w.dt))
        az = thrust - 1.0
        assert abs(traj[-1, 2] - (0.5 + az * t * t / 2)) < 1e-12
        assert abs(traj[-1, 8] - az * t) < 1e-12


def test_quadrotor_rk4_order(kpo):
    """Generic tumbling motion: RK4's global error falls ~16x per halving."""
    w = W.c3(0)
    x0 = np.array([0.5, 0.5, 0.5, 0.1, -0.1, 0.3, 0.05, 0.0, -0.05, 0.5, -0.4, 0.3])
    u = [0.31, 0.22, 0.27, 0.18]
    ref = x0.copy()
    for _ in range(1600):
        ref = kpo.step(w, ref, u, 1.0 / 1600)
    errs = []
    for n in (25, 50, 100):
        x = x0.copy()
        for _ in range(n):
            x = kpo.step(w, x, u, 1.0 / n)
        errs.append(np.linalg.norm(x - ref))
    for a, b in zip(errs, errs[1:]):
        assert 12.0 < a / b < 20.0
