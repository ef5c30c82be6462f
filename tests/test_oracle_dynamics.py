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


def _rx(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])


def _ry(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])


def _rz(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])


def _attitude(phi, theta, psi):
    """Body-to-world rotation of ZYX Euler angles: yaw, then pitch, then roll."""
    return _rz(psi) @ _ry(theta) @ _rx(phi)


def _hat(w):
    return np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])


def _rotation_exp(w, t):
    """exp(t [w]x) by Rodrigues' formula."""
    n = np.linalg.norm(w)
    K = _hat(np.asarray(w) / n)
    a = n * t
    return np.eye(3) + math.sin(a) * K + (1 - math.cos(a)) * K @ K


def test_quadrotor_tilted_thrust_follows_the_rotation_matrix(kpo):
    """Equal rotor thrusts and no body rates: no torque, so the attitude holds
    and the acceleration is the constant R(phi, theta, psi) e3 F / m - g e3,
    with R built from elementary rotations; positions are then exact
    parabolas under RK4."""
    w = W.c3(0)
    rng = np.random.default_rng(3)
    for _ in range(12):
        phi, theta, psi = rng.uniform(-0.6, 0.6), rng.uniform(-0.6, 0.6), rng.uniform(-3, 3)
        F = rng.uniform(0.2, 1.8)
        x0 = np.zeros(12)
        x0[:3] = rng.uniform(0.3, 0.7, 3)
        x0[3:6] = (phi, theta, psi)
        x0[6:9] = rng.uniform(-0.2, 0.2, 3)
        a = _attitude(phi, theta, psi) @ np.array([0.0, 0.0, F]) - np.array([0.0, 0.0, 1.0])
        k = 30
        t = k * float(np.float32(w.dt))
        traj = kpo.propagate(w, x0, [F / 4] * 4, k)
        np.testing.assert_allclose(traj[-1, 6:9], x0[6:9] + a * t, atol=1e-12)
        np.testing.assert_allclose(traj[-1, :3], x0[:3] + x0[6:9] * t + a * t * t / 2, atol=1e-12)
        np.testing.assert_allclose(traj[-1, 3:6], x0[3:6], atol=1e-14)
        np.testing.assert_allclose(traj[-1, 9:], 0.0, atol=1e-14)


def test_quadrotor_body_rates_turn_the_attitude(kpo):
    """Constant body rates (torque free: (p, q, 0), or (0, 0, r), with
    Ixx = Iyy) turn the attitude as R(t) = R(0) exp(t [omega]x); the Euler
    angles integrated by the oracle must give that rotation."""
    w = W.c3(0)
    assert W.QUAD_PHYS["Ixx"] == W.QUAD_PHYS["Iyy"]
    rng = np.random.default_rng(4)
    for omega in ([0.6, -0.4, 0.0], [0.0, 0.0, 0.9], [-0.3, 0.5, 0.0]):
        for _ in range(3):
            eta0 = (rng.uniform(-0.4, 0.4), rng.uniform(-0.4, 0.4), rng.uniform(-2, 2))
            x = np.zeros(12)
            x[:3] = 0.5
            x[3:6] = eta0
            x[9:] = omega
            n, t = 500, 0.5
            for _ in range(n):
                x = kpo.step(w, x, [0.25] * 4, t / n)
            np.testing.assert_allclose(x[9:], omega, atol=1e-12)
            want = _attitude(*eta0) @ _rotation_exp(omega, t)
            np.testing.assert_allclose(_attitude(*x[3:6]), want, atol=1e-10)


def test_quadrotor_rotor_torques_and_gyroscopic_coupling(kpo):
    """Roll torque l (T2 - T4) and pitch torque l (T3 - T1) from rest give
    p = 2 l d t / Ixx and q = 2 l e t / Iyy; torque free, a symmetric body
    (Ixx = Iyy = I1, Izz = I3) precesses its (p, q) at
    Omega = (I3 - I1) r / I1 (Euler's equations)."""
    w = W.c3(0)
    # the constants as the workload stores them (float32)
    P = {k: float(np.float32(v)) for k, v in W.QUAD_PHYS.items()}
    T0, d = 0.25, 0.03
    k = 20
    t = k * float(np.float32(w.dt))
    x0 = np.zeros(12)
    x0[:3] = 0.5
    roll = kpo.propagate(w, x0, [T0, T0 + d, T0, T0 - d], k)[-1]
    assert abs(roll[9] - 2 * P["l"] * d * t / P["Ixx"]) < 1e-12
    assert abs(roll[10]) < 1e-14 and abs(roll[11]) < 1e-14
    pitch = kpo.propagate(w, x0, [T0 - d, T0, T0 + d, T0], k)[-1]
    assert abs(pitch[10] - 2 * P["l"] * d * t / P["Iyy"]) < 1e-12
    assert abs(pitch[9]) < 1e-14 and abs(pitch[11]) < 1e-14
    # torque-free precession
    p0, q0, r0 = 0.4, -0.3, 0.8
    x = x0.copy()
    x[9:] = (p0, q0, r0)
    n, T = 400, 2.0
    for _ in range(n):
        x = kpo.step(w, x, [T0] * 4, T / n)
    Om = (P["Izz"] - P["Ixx"]) * r0 / P["Ixx"]
    want = (p0 * math.cos(Om * T) - q0 * math.sin(Om * T),
            p0 * math.sin(Om * T) + q0 * math.cos(Om * T), r0)
    np.testing.assert_allclose(x[9:], want, atol=1e-10)
