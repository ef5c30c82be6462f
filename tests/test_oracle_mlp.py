"""Pins of the oracle's learned-proposal network and draw (an addition to
the paper's uniform control draw in Algorithm 2)."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import kpo
from oracle.kpo import Oracle
from paper_2409_06807_gb300 import workloads as W


def _params(seed, scale=0.2):
    rng = np.random.default_rng(seed)
    return rng.normal(0, scale, kpo.mlp_num_params())


def _batch(seed, m=6):
    rng = np.random.default_rng(seed)
    x = np.zeros((m, 32))
    x[:, :20] = rng.normal(0, 1, (m, 20))
    t = rng.uniform(-0.9, 0.9, (m, 4))
    return x, t


def test_parameter_count():
    assert kpo.mlp_num_params() == 256 * 32 + 256 + 256 * 256 + 256 + 8 * 256 + 8


def test_finite_difference_gradient():
    """Backpropagation against central differences in FP64 on a sample of
    coordinates of every parameter block."""
    p = _params(1)
    x, t = _batch(2)
    loss, g = kpo.mlp_loss_grad(p, x, t)
    rng = np.random.default_rng(3)
    offsets = np.cumsum([0, 256 * 32, 256, 256 * 256, 256, 8 * 256, 8])
    for b in range(6):
        for i in rng.integers(offsets[b], offsets[b + 1], 12):
            h = 1e-6
            pp, pm = p.copy(), p.copy()
            pp[i] += h
            pm[i] -= h
            fd = (kpo.mlp_loss_grad(pp, x, t, False)[0] - kpo.mlp_loss_grad(pm, x, t, False)[0]) / (2 * h)
            assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (b, i, fd, g[i])


def test_forward_special_cases():
    """Zero weights: the outputs are the heads of the last bias; a target
    equal to the mean with unit std gives zero loss."""
    p = np.zeros(kpo.mlp_num_params())
    W1, b1, W2, b2, W3, b3 = kpo.mlp_split(p)
    b3[:] = [0.3, -0.2, 0.0, 2.0, 0.0, -7.0, 5.0, -0.5]
    x, _ = _batch(4, 3)
    out = kpo.mlp_forward(p, x)
    np.testing.assert_allclose(out[:, :4], np.tanh(b3[:4])[None].repeat(3, 0), atol=1e-15)
    np.testing.assert_allclose(out[:, 4:], np.array([[0.0, -4.0, 1.0, -0.5]] * 3), atol=0)
    b3[4:] = 0.0
    t = np.tanh(b3[:4])[None].repeat(3, 0)
    loss, _ = kpo.mlp_loss_grad(p, x, t)
    assert abs(loss) < 1e-15


def test_relu_layer_by_hand():
    """One active unit per layer: out = tanh(w3 * relu(w2 * relu(w1 . x)))."""
    p = np.zeros(kpo.mlp_num_params())
    W1, b1, W2, b2, W3, b3 = kpo.mlp_split(p)
    W1[5, 2] = 0.5
    W2[7, 5] = 2.0
    W3[1, 7] = -0.25
    x = np.zeros((2, 32))
    x[0, 2], x[1, 2] = 3.0, -3.0
    out = kpo.mlp_forward(p, x)
    assert math.isclose(out[0, 1], math.tanh(-0.25 * 2.0 * 1.5), rel_tol=1e-15)
    assert out[1, 1] == 0.0  # the ReLU cut the negative input


def test_adam_first_step_is_sign_step():
    """Adam's bias-corrected first step moves every coordinate by lr times
    the sign of its gradient (up to eps)."""
    p = np.ones(10)
    g = np.linspace(-2, 2, 10)
    g[5] = 0.5
    m, v = np.zeros(10), np.zeros(10)
    kpo.adam(p, g, m, v, 0.01, 1)
    np.testing.assert_allclose(p, 1 - 0.01 * np.sign(g), atol=1e-7)


def test_box_muller_normals():
    rng = np.random.default_rng(0)
    z = np.concatenate([kpo.box_muller(rng.integers(0, 2 ** 32, 4, dtype=np.uint64).astype(np.uint32))
                        for _ in range(4000)])
    assert stats.kstest(z, "norm").pvalue > 1e-4
    assert np.all(np.isfinite(kpo.box_muller(np.zeros(4, np.uint32))))


def test_features_by_hand():
    """Node features of the root of a tiny double-integrator query."""
    w = W.tiny(W.DI)
    o = Oracle(w)
    o.reset()
    f = o.features(0)
    x = w.x_init.astype(np.float64)
    np.testing.assert_allclose(f[:3], 2 * x[:3] - 1, atol=1e-15)
    np.testing.assert_allclose(f[3:6], 0.0, atol=1e-15)  # zero velocity mid-range
    np.testing.assert_allclose(f[6:9], w.goal_c - x[:3], atol=1e-7)
    assert f[9] == 1 / 8  # one visited sub-region of 8
    assert f[10] == 1.0 and f[11] == 0.0 and f[12] == 0.0 and f[13] == 1.0
    # root in region (0,0,1) of 2^3: neighbours +x, +y and -z exist (P = 1)
    np.testing.assert_array_equal(f[14:20], [0, 1, 0, 1, 1, 0])
    assert np.all(f[20:] == 0)


def test_learned_draw_and_harvest():
    """With a network, a mixed fraction of samples follows its Gaussian;
    the harvest collects exactly the representatives of new sub-regions."""
    w = W.c1(0)
    o = Oracle(w)
    o.reset()
    p = np.zeros(kpo.mlp_num_params(), np.float32)
    _, _, _, _, _, b3 = kpo.mlp_split(p)
    b3[:] = [0.0, 0.0, 0.0, 0.0, -4.0, -4.0, -4.0, -4.0]  # narrow, centred
    o.set_mlp(p, mix=0.5)
    o.set_harvest(100000)
    o.run(2)
    _, st, rec = o.iterate(records=True)
    u = rec["uraw"]
    sel = np.array([kpo.philox4x32_10([st["iteration"], n, k % st["lambda"], 1],
                                      [w.seed & 0xFFFFFFFF, w.seed >> 32])[2]
                    for k, n in enumerate(rec["node"])])
    learned = sel < 2 ** 31
    assert 0.4 < learned.mean() < 0.6
    # every duration, learned or not, is the uniform draw of purpose 1
    kw = np.array([kpo.philox4x32_10([st["iteration"], n, k % st["lambda"], 1],
                                     [w.seed & 0xFFFFFFFF, w.seed >> 32])[0]
                   for k, n in enumerate(rec["node"])], np.uint64)
    span = w.k_max - w.k_min + 1
    assert np.array_equal(rec["k"], w.k_min + ((kw * span) >> 32).astype(np.int64))
    # learned controls sit at the middle of U (narrow Gaussians centred at
    # 0): the pass's new nodes follow its accepted keys in order
    t = o.export()
    acc = np.flatnonzero(rec["flags"] & 16)
    ctrl = t["ctrl"][t["n_nodes"] - len(acc):]
    lo, hi = np.asarray(w.u_lo[:3], np.float64), np.asarray(w.u_hi[:3], np.float64)
    q = 2 * (ctrl - lo) / (hi - lo) - 1
    lrn = learned[acc]
    assert lrn.any() and (~lrn).any()
    assert np.max(np.abs(q[lrn])) < 0.2
    assert np.max(np.abs(q[~lrn])) > 0.5
    hf, ht = o.harvest()
    assert len(hf) > 0 and np.all(np.abs(ht) <= 1.0 + 1e-12)
