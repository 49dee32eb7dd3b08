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
