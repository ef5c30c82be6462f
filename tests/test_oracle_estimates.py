"""Pins of Eq. 3-5 (Algorithm 3) and Eq. 6 in the oracle."""
import math

import numpy as np

from conftest import read_golden


def test_worked_example(kpo):
    g = {k: float(v) for k, v in read_golden("eq345_worked_example.txt")}
    score, p, thr, s = kpo.eq345([3, 0, 5, 0], [1, 0, 5, 7], [2, 1, 0, 1],
                                 [1, 1, 0, 1], 1 / 8, 1.0, 0.01)
    for i in range(4):
        assert math.isclose(score[i], g[f"score{i}"], rel_tol=1e-15, abs_tol=0)
        assert math.isclose(p[i], g[f"p{i}"], rel_tol=1e-15)
    assert math.isclose(s, g["sum"], rel_tol=1e-15)


def test_probability_mass_and_lemma1(kpo):
    """Without clipping, sum over R_avail of P = 1 + eps |R_avail| (the
    normalised scores sum to one); P >= eps always (Lemma 1); regions
    outside R_avail keep P = 1; thr brackets P on the 2^-32 grid."""
    rng = np.random.default_rng(0)
    for trial in range(50):
        n = int(rng.integers(1, 300))
        nv = rng.integers(0, 1000, n)
        ni = rng.integers(0, 1000, n)
        cov = rng.integers(0, 64, n)
        avail = (rng.random(n) < 0.7).astype(np.uint8)
        eps = 10.0 ** rng.uniform(-4, -1)
        score, p, thr, s = kpo.eq345(nv, ni, cov, avail, 0.01, 1.0, eps)
        a = avail == 1
        assert np.all(p[~a] == 1.0) and np.all(score[~a] == 0.0)
        assert np.all(p[a] >= eps) and np.all(p <= 1.0)
        if a.any() and np.all(p[a] < 1.0):
            assert math.isclose(p[a].sum(), 1.0 + eps * a.sum(), rel_tol=1e-12)
        assert math.isclose(s, math.fsum(score), rel_tol=1e-13)
        t = thr.astype(np.float64) / 2.0 ** 32
        assert np.all(t <= p) and np.all(p < t + 2.0 ** -32 + (p == 1.0))


def test_score_monotonicity(kpo):
    """Score falls with coverage and with sample count; FreeVol equals the
    region volume when no sample was invalid."""
    base, _, _, _ = kpo.eq345([10], [5], [3], [1], 0.5, 1.0, 0.01)
    more_cov, _, _, _ = kpo.eq345([10], [5], [4], [1], 0.5, 1.0, 0.01)
    more_inv, _, _, _ = kpo.eq345([10], [6], [3], [1], 0.5, 1.0, 0.01)
    assert more_cov[0] < base[0] and more_inv[0] < base[0]
    s, _, _, _ = kpo.eq345([7], [0], [0], [1], 0.5, 1.0, 0.01)
    assert math.isclose(s[0], 0.5 ** 4 / (1 * (1 + 49)), rel_tol=1e-15)


def test_lambda_eq6_floor_property(kpo):
    """lambda = min(lambda_max, floor((t_e - |T|)/|V_E|)) characterised by
    lambda |V_E| <= t_e - |T| < (lambda + 1) |V_E| unless capped."""
    rng = np.random.default_rng(2)
    for _ in range(2000):
        t_e = int(rng.integers(1, 1 << 22))
        n = int(rng.integers(1, t_e + 1))
        ve = int(rng.integers(1, n + 1))
        lm = int(rng.integers(1, 256))
        lam = kpo.lam(t_e, n, ve, lm)
        room = t_e - n
        assert 0 <= lam <= lm and lam * ve <= room
        assert lam == lm or (lam + 1) * ve > room
