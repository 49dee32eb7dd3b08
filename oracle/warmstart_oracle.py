"""FP64 CPU oracle of the warm-start network (forward pass, loss and gradients).

TEST INFRASTRUCTURE ONLY: used by the tests to check the network kernels; the product path never
imports it.  Plain numpy, obvious loops over the nine taps; the backward pass is the chain rule
written out layer by layer.  Layouts as in the C ABI: activations (B, H, W, C); 32->32 weights
(co, tap, ci) with tap = 3 dy + dx; input-layer weights (co, tap); output-layer weights (tap, ci);
"same" zero padding.
"""
from __future__ import annotations

import numpy as np

OFFS = [(t // 3 - 1, t % 3 - 1) for t in range(9)]


def shift(x, dy, dx):
    """y[b, i, j] = x[b, i + dy, j + dx] (zero outside)."""
    B, H, W = x.shape[:3]
    y = np.zeros_like(x)
    ys, ye = max(0, -dy), min(H, H - dy)
    xs, xe = max(0, -dx), min(W, W - dx)
    y[:, ys:ye, xs:xe] = x[:, ys + dy:ye + dy, xs + dx:xe + dx]
    return y


def conv(x, w, b=None):
    """x (B,H,W,Cin), w (Cout, 9, Cin) -> (B,H,W,Cout): sum_tap x[p + off(tap)] . w[:, tap, :]^T + b."""
    y = sum(shift(x, dy, dx) @ w[:, t, :].T for t, (dy, dx) in enumerate(OFFS))
    return y + (0.0 if b is None else b)


def conv_backward(x, w, dy):
    """Gradients of conv: dx, dw, db for upstream gradient dy."""
    dx = sum(shift(dy @ w[:, t, :], -oy, -ox) for t, (oy, ox) in enumerate(OFFS))
    dw = np.stack([np.einsum("bhwo,bhwi->oi", dy, shift(x, oy, ox)) for (oy, ox) in OFFS], axis=1)
    return dx, dw, dy.sum(axis=(0, 1, 2))


def pool2(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def up2(x):
    return x.repeat(2, axis=1).repeat(2, axis=2)


class Net:
    """Parameters: w1 (32, 9) b1 (32); w2..w5 (32, 9, 32) b2..b5 (32); w6 (9, 32) b6 (1)."""

    def __init__(self, params: dict):
        self.p = {k: np.asarray(v, np.float64) for k, v in params.items()}

    def forward(self, x0):
        p = self.p
        c = {"x0": x0}
        c["a1"] = np.maximum(conv(x0[..., None], p["w1"][:, :, None], p["b1"]), 0)
        c["a2"] = np.maximum(conv(c["a1"], p["w2"], p["b2"]), 0)
        c["p2"] = pool2(c["a2"])
        c["a3"] = np.maximum(conv(c["p2"], p["w3"], p["b3"]), 0)
        c["a4"] = np.maximum(conv(c["a3"], p["w4"], p["b4"]), 0)
        c["s5"] = up2(c["a4"]) + c["a2"]
        c["a5"] = np.maximum(conv(c["s5"], p["w5"], p["b5"]), 0)
        c["z"] = conv(c["a5"], p["w6"][None], p["b6"])[..., 0]
        self.cache = c
        return c["z"]

    def loss_and_grads(self, x0, t):
        z = self.forward(x0)
        c, p = self.cache, self.p
        n = z.size
        loss = float(np.sum((z - t) ** 2))
        dz = 2.0 * (z - t) / n
        g = {}
        da5, dw6, db6 = conv_backward(c["a5"], p["w6"][None], dz[..., None])
        g["w6"], g["b6"] = dw6[0], db6
        dz5 = da5 * (c["a5"] > 0)
        ds5, g["w5"], g["b5"] = conv_backward(c["s5"], p["w5"], dz5)
        dz4 = pool2(ds5) * 4.0 * (c["a4"] > 0)          # up^T = sum over each 2x2 block
        da3, g["w4"], g["b4"] = conv_backward(c["a3"], p["w4"], dz4)
        dz3 = da3 * (c["a3"] > 0)
        dp2, g["w3"], g["b3"] = conv_backward(c["p2"], p["w3"], dz3)
        dz2 = (ds5 + up2(dp2) / 4.0) * (c["a2"] > 0)
        da1, g["w2"], g["b2"] = conv_backward(c["a1"], p["w2"], dz2)
        dz1 = da1 * (c["a1"] > 0)
        _, dw1, g["b1"] = conv_backward(x0[..., None], p["w1"][:, :, None], dz1)
        g["w1"] = dw1[:, :, 0]
        return loss, g


def adam(p, g_steps, lr, b1=0.9, b2=0.999, eps=1e-8):
    """Adam (Kingma and Ba) on parameters p for the gradient sequence g_steps: moments
    m = b1 m + (1 - b1) g and v = b2 v + (1 - b2) g^2, bias-corrected m / (1 - b1^t) and
    v / (1 - b2^t), step p -= lr m_hat / (sqrt(v_hat) + eps), t = 1, 2, ...  Returns (p, m, v)."""
    p = np.array(p, np.float64, copy=True)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for t, g in enumerate(g_steps, start=1):
        g = np.asarray(g, np.float64)
        m = b1 * m + (1.0 - b1) * g
        v = b2 * v + (1.0 - b2) * g * g
        mh = m / (1.0 - b1 ** t)
        vh = v / (1.0 - b2 ** t)
        p = p - lr * mh / (np.sqrt(vh) + eps)
    return p, m, v
