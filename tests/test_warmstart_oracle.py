"""Pins of the FP64 warm-start network oracle (CPU): the convolution against scipy's correlate, and
every parameter gradient against central finite differences of the loss."""
import numpy as np
from scipy import signal

from oracle import warmstart_oracle as WO


def _params(rng, scale=0.3):
    p = {"w1": rng.standard_normal((32, 9)) * scale, "b1": rng.standard_normal(32) * 0.1,
         "w6": rng.standard_normal((9, 32)) * 0.1, "b6": rng.standard_normal(1) * 0.1}
    for i in range(2, 6):
        p[f"w{i}"] = rng.standard_normal((32, 9, 32)) * 0.1
        p[f"b{i}"] = rng.standard_normal(32) * 0.1
    return p


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 12, 10, 3))
    w = rng.standard_normal((2, 9, 3))
    y = WO.conv(x, w)
    for co in range(2):
        ref = sum(signal.correlate2d(x[0, :, :, ci], w[co, :, ci].reshape(3, 3), mode="same") for ci in range(3))
        np.testing.assert_allclose(y[0, :, :, co], ref, atol=1e-12)


def test_network_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    p = _params(rng)
    x0 = rng.standard_normal((2, 8, 8))
    t = rng.standard_normal((2, 8, 8))
    net = WO.Net(p)
    _, g = net.loss_and_grads(x0, t)
    for name in p:
        flat = net.p[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
            old = flat[idx]
            h = 1e-6
            flat[idx] = old + h
            lp, _ = net.loss_and_grads(x0, t)
            flat[idx] = old - h
            lm, _ = net.loss_and_grads(x0, t)
            flat[idx] = old
            fd = (lp - lm) / (2 * h) / x0.size
            an = g[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 + 1e-5 * abs(fd), (name, idx, fd, an)


def test_adam_first_steps_closed_form():
    """After one step the bias-corrected moments are g and g^2, so each parameter moves by
    lr g / (|g| + eps), i.e. lr sign(g) up to eps; with a constant gradient every step moves by the
    same amount; with g then -g the second step follows the hand-worked moments."""
    p0 = np.array([1.0, -2.0, 0.5, 3.0])
    g = np.array([0.3, -4.0, 1e-3, 0.0])
    lr, eps = 0.01, 1e-8
    p1, m1, v1 = WO.adam(p0, [g], lr, eps=eps)
    np.testing.assert_allclose(p1, p0 - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-12)
    np.testing.assert_allclose(v1, 0.001 * g * g, rtol=1e-12)
    pc, _, _ = WO.adam(p0, [g] * 5, lr, eps=eps)
    np.testing.assert_allclose(pc, p0 - 5 * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-12)
    p2, m2, v2 = WO.adam(p0, [g, -g], lr, b1=0.9, b2=0.999, eps=eps)
    m_hand = 0.9 * 0.1 * g - 0.1 * g            # 0.09 g - 0.1 g = -0.01 g
    v_hand = 0.999 * 0.001 * g * g + 0.001 * g * g
    step2 = lr * (m_hand / (1 - 0.81)) / (np.sqrt(v_hand / (1 - 0.999 ** 2)) + eps)
    np.testing.assert_allclose(m2, m_hand, rtol=1e-12)
    np.testing.assert_allclose(p2, p1 - step2, rtol=0, atol=1e-14)
