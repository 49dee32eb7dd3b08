"""Learned warm start for SGP: a small BF16 convolutional encoder-decoder that predicts f^(0) from g.

Architecture, layouts and kernels: include/warmstart.h.  This module only allocates tensors
(PyTorch supplies device memory), marshals arguments and sequences the library kernels; every
numeric step (convolutions, their gradients, pooling, loss, Adam, normalisation, the SGP solves that
produce the training targets) runs in the library.  SGP always refines the predicted start to the
same stopping rule as the flat start.
"""
from __future__ import annotations

import ctypes as C
import math
import time

import numpy as np

from . import scenes
from . import sgp as lib

PARAMS = [("w1", 32 * 9), ("b1", 32)] + \
    [(f"{k}{i}", n) for i in range(2, 6) for k, n in (("w", 32 * 9 * 32), ("b", 32))] + [("w6", 9 * 32), ("b6", 1)]
CONV32 = ["w2", "w3", "w4", "w5"]

_ws = None


def _lib():
    global _ws
    if _ws is not None:
        return _ws
    L = lib.load()
    vp, i, sz, f = C.c_void_p, C.c_int, C.c_size_t, C.c_float
    sig = {
        "ws_conv32": [vp, vp, vp, vp, vp, i, i, i, i, vp],
        "ws_conv32_wgrad": [vp, vp, vp, i, i, i, vp],
        "ws_flip_weights": [vp, vp, vp],
        "ws_conv_in": [vp, vp, vp, vp, i, i, i, vp],
        "ws_conv_out": [vp, vp, vp, vp, i, i, i, vp],
        "ws_conv_out_dgrad": [vp, vp, vp, vp, i, i, i, vp],
        "ws_small_wgrad": [vp, vp, vp, vp, i, i, i, i, vp],
        "ws_bias_grad": [vp, vp, i, i, i, vp],
        "ws_pool2": [vp, vp, i, i, i, vp],
        "ws_up2_add": [vp, vp, vp, i, i, i, vp],
        "ws_junction_bwd": [vp, vp, vp, vp, i, i, i, vp],
        "ws_up2_bwd_mask": [vp, vp, vp, i, i, i, vp],
        "ws_loss": [vp, vp, vp, vp, sz, vp],
        "ws_adam": [vp, vp, vp, vp, i, f, f, f, f, i, vp],
        "ws_to_bf16": [vp, vp, i, vp],
        "ws_prep": [vp, vp, vp, vp, vp, vp, i, sz, vp],
        "ws_start": [vp, vp, vp, vp, i, sz, vp],
        "ws_scale": [vp, vp, vp, i, sz, vp],
        "ws_zero": [vp, sz, vp],
        "ws_error": [C.POINTER(C.c_int)],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.restype = C.c_int
        fn.argtypes = args
    _ws = L
    return L


def _ok(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"{what} failed with code {rc}")


def device_error() -> int:
    """Read and clear the device-side error flag of the warm-start kernels (ws_error)."""
    v = C.c_int()
    _ok(_lib().ws_error(C.byref(v)), "ws_error")
    return v.value


def _p(t):
    return None if t is None else t.data_ptr()


class WarmStartNet:
    """Parameters live in one FP32 buffer (master copy) with Adam moments and a gradient buffer;
    the 32 -> 32 layers also keep bf16 working copies and their flipped (transposed) copies."""

    def __init__(self, seed: int = 0, device: str = "cuda"):
        import torch
        self.torch = torch
        self.dev = torch.device(device)
        self.off = {}
        o = 0
        for name, n in PARAMS:
            self.off[name] = (o, n)
            o += n
        self.n = o
        rng = np.random.default_rng(seed)
        host = np.zeros(o, np.float32)
        for name, n in PARAMS:
            a, _ = self.off[name]
            if name.startswith("w"):
                fan_in = 9 if name == "w1" else 288
                std = math.sqrt(2.0 / fan_in) * (0.1 if name == "w6" else 1.0)
                host[a:a + n] = rng.standard_normal(n) * std
        self.p = torch.from_numpy(host).to(self.dev)
        self.g = torch.zeros(o, dtype=torch.float32, device=self.dev)
        self.m = torch.zeros_like(self.g)
        self.v = torch.zeros_like(self.g)
        self.wb = {k: torch.empty(32 * 9 * 32, dtype=torch.bfloat16, device=self.dev) for k in CONV32}
        self.wt = {k: torch.empty(32 * 9 * 32, dtype=torch.bfloat16, device=self.dev) for k in CONV32}
        self.t = 0
        self._bufs = {}
        self.sync_weights()

    # ------------------------------------------------------------------ helpers
    def stream(self):
        return self.torch.cuda.current_stream().cuda_stream

    def view(self, buf, name):
        a, n = self.off[name]
        return buf[a:a + n]

    def set_params(self, params: dict) -> None:
        """Load parameters given as numpy arrays in the layouts of include/warmstart.h."""
        host = self.p.cpu().numpy()
        for name, arr in params.items():
            a, n = self.off[name]
            host[a:a + n] = np.asarray(arr, np.float32).reshape(-1)
        self.p.copy_(self.torch.from_numpy(host))
        self.sync_weights()

    def params(self) -> dict:
        host = self.p.cpu().numpy()
        return {name: host[a:a + n].copy() for name, (a, n) in self.off.items()}

    def sync_weights(self) -> None:
        L, s = _lib(), self.stream()
        for k in CONV32:
            _ok(L.ws_to_bf16(_p(self.view(self.p, k)), _p(self.wb[k]), 32 * 288, s), "to_bf16")
            _ok(L.ws_flip_weights(_p(self.wb[k]), _p(self.wt[k]), s), "flip")

    def buffers(self, B, H, W):
        key = (B, H, W)
        if key not in self._bufs:
            t, d = self.torch, self.dev
            full = (B, H, W, 32)
            half = (B, H // 2, W // 2, 32)
            bf = t.bfloat16
            self._bufs[key] = dict(
                x0=t.empty((B, H, W), dtype=t.float32, device=d), tgt=t.empty((B, H, W), dtype=t.float32, device=d),
                s=t.empty(B, dtype=t.float32, device=d), b=t.empty(B, dtype=t.float32, device=d),
                a1=t.empty(full, dtype=bf, device=d), a2=t.empty(full, dtype=bf, device=d),
                p2=t.empty(half, dtype=bf, device=d), a3=t.empty(half, dtype=bf, device=d),
                a4=t.empty(half, dtype=bf, device=d), s5=t.empty(full, dtype=bf, device=d),
                a5=t.empty(full, dtype=bf, device=d), z=t.empty((B, H, W), dtype=t.float32, device=d),
                dz=t.empty((B, H, W), dtype=t.float32, device=d), d5=t.empty(full, dtype=bf, device=d),
                ds5=t.empty(full, dtype=bf, device=d), dz4=t.empty(half, dtype=bf, device=d),
                dz3=t.empty(half, dtype=bf, device=d), dp2=t.empty(half, dtype=bf, device=d),
                dz2=t.empty(full, dtype=bf, device=d), dz1=t.empty(full, dtype=bf, device=d),
                loss=t.zeros(1, dtype=t.float64, device=d))
        return self._bufs[key]

    # ------------------------------------------------------------------ passes
    def prepare(self, g, b, f=None):
        """x0 = (g - b)/s and (with f) the training target; g, f (B, H, W) fp32 CUDA, b (B,) fp32 CUDA."""
        L, s = _lib(), self.stream()
        B, H, W = g.shape
        bf = self.buffers(B, H, W)
        bf["b"].copy_(b)
        _ok(L.ws_scale(_p(g), _p(bf["b"]), _p(bf["s"]), B, H * W, s), "scale")
        _ok(L.ws_prep(_p(g), _p(f), _p(bf["b"]), _p(bf["s"]), _p(bf["x0"]), _p(bf["tgt"]), B, H * W, s), "prep")
        return bf

    def forward(self, bf, B, H, W):
        L, s, P = _lib(), self.stream(), self.p
        v = lambda k: _p(self.view(P, k))
        _ok(L.ws_conv_in(_p(bf["x0"]), v("w1"), v("b1"), _p(bf["a1"]), B, H, W, s), "conv_in")
        _ok(L.ws_conv32(_p(bf["a1"]), _p(self.wb["w2"]), v("b2"), None, _p(bf["a2"]), B, H, W, 0, s), "conv2")
        _ok(L.ws_pool2(_p(bf["a2"]), _p(bf["p2"]), B, H, W, s), "pool")
        _ok(L.ws_conv32(_p(bf["p2"]), _p(self.wb["w3"]), v("b3"), None, _p(bf["a3"]), B, H // 2, W // 2, 0, s), "conv3")
        _ok(L.ws_conv32(_p(bf["a3"]), _p(self.wb["w4"]), v("b4"), None, _p(bf["a4"]), B, H // 2, W // 2, 0, s), "conv4")
        _ok(L.ws_up2_add(_p(bf["a4"]), _p(bf["a2"]), _p(bf["s5"]), B, H, W, s), "up")
        _ok(L.ws_conv32(_p(bf["s5"]), _p(self.wb["w5"]), v("b5"), None, _p(bf["a5"]), B, H, W, 0, s), "conv5")
        _ok(L.ws_conv_out(_p(bf["a5"]), v("w6"), v("b6"), _p(bf["z"]), B, H, W, s), "conv_out")
        return bf["z"]

    def backward(self, bf, B, H, W):
        """Accumulate parameter gradients of the loss (dz in bf['dz']) into self.g."""
        L, s, P, G = _lib(), self.stream(), self.p, self.g
        v = lambda buf, k: _p(self.view(buf, k))
        h, w = H // 2, W // 2
        _ok(L.ws_small_wgrad(_p(bf["dz"]), _p(bf["a5"]), v(G, "w6"), v(G, "b6"), B, H, W, 1, s), "wgrad6")
        _ok(L.ws_conv_out_dgrad(_p(bf["dz"]), v(P, "w6"), _p(bf["a5"]), _p(bf["d5"]), B, H, W, s), "dgrad6")
        # layer 5: input s5, output gradient dz5 = d5
        _ok(L.ws_conv32_wgrad(_p(bf["d5"]), _p(bf["s5"]), v(G, "w5"), B, H, W, s), "wgrad5")
        _ok(L.ws_bias_grad(_p(bf["d5"]), v(G, "b5"), B, H, W, s), "bgrad5")
        _ok(L.ws_conv32(_p(bf["d5"]), _p(self.wt["w5"]), None, None, _p(bf["ds5"]), B, H, W, 3, s), "dgrad5")
        _ok(L.ws_up2_bwd_mask(_p(bf["ds5"]), _p(bf["a4"]), _p(bf["dz4"]), B, H, W, s), "upbwd")
        # layer 4 (half resolution): input a3
        _ok(L.ws_conv32_wgrad(_p(bf["dz4"]), _p(bf["a3"]), v(G, "w4"), B, h, w, s), "wgrad4")
        _ok(L.ws_bias_grad(_p(bf["dz4"]), v(G, "b4"), B, h, w, s), "bgrad4")
        _ok(L.ws_conv32(_p(bf["dz4"]), _p(self.wt["w4"]), None, _p(bf["a3"]), _p(bf["dz3"]), B, h, w, 2, s), "dgrad4")
        # layer 3: input p2
        _ok(L.ws_conv32_wgrad(_p(bf["dz3"]), _p(bf["p2"]), v(G, "w3"), B, h, w, s), "wgrad3")
        _ok(L.ws_bias_grad(_p(bf["dz3"]), v(G, "b3"), B, h, w, s), "bgrad3")
        _ok(L.ws_conv32(_p(bf["dz3"]), _p(self.wt["w3"]), None, None, _p(bf["dp2"]), B, h, w, 3, s), "dgrad3")
        _ok(L.ws_junction_bwd(_p(bf["ds5"]), _p(bf["dp2"]), _p(bf["a2"]), _p(bf["dz2"]), B, H, W, s), "junction")
        # layer 2: input a1
        _ok(L.ws_conv32_wgrad(_p(bf["dz2"]), _p(bf["a1"]), v(G, "w2"), B, H, W, s), "wgrad2")
        _ok(L.ws_bias_grad(_p(bf["dz2"]), v(G, "b2"), B, H, W, s), "bgrad2")
        _ok(L.ws_conv32(_p(bf["dz2"]), _p(self.wt["w2"]), None, _p(bf["a1"]), _p(bf["dz1"]), B, H, W, 2, s), "dgrad2")
        # layer 1: input x0
        _ok(L.ws_small_wgrad(_p(bf["dz1"]), _p(bf["x0"]), v(G, "w1"), v(G, "b1"), B, H, W, 0, s), "wgrad1")

    def loss_and_grad(self, bf, B, H, W) -> None:
        L, s = _lib(), self.stream()
        _ok(L.ws_zero(_p(self.g), self.n * 4, s), "zero")
        _ok(L.ws_zero(_p(bf["loss"]), 8, s), "zero")
        self.forward(bf, B, H, W)
        _ok(L.ws_loss(_p(bf["z"]), _p(bf["tgt"]), _p(bf["dz"]), _p(bf["loss"]), B * H * W, s), "loss")
        self.backward(bf, B, H, W)

    def adam(self, lr: float) -> None:
        self.t += 1
        _ok(_lib().ws_adam(_p(self.p), _p(self.m), _p(self.v), _p(self.g), self.n, lr, 0.9, 0.999, 1e-8, self.t,
                           self.stream()), "adam")
        self.sync_weights()

    def predict(self, g, b):
        """f0 (B, H, W) fp32 for detected images g (B, H, W) with backgrounds b (B,)."""
        B, H, W = g.shape
        bf = self.prepare(g, b)
        self.forward(bf, B, H, W)
        f0 = self.torch.empty_like(g)
        _ok(_lib().ws_start(_p(bf["z"]), _p(bf["x0"]), _p(bf["s"]), _p(f0), B, H * W, self.stream()), "start")
        return f0


# ---------------------------------------------------------------------- data, training, evaluation
def make_scenes(n: int, N: int, seed: int):
    rng = scenes.rng_for(seed)
    return [scenes.warmstart_scene(rng, N) for _ in range(n)]


def sgp_solutions(scs, max_iter: int = 400, batch: int = 64):
    """SGP from the flat start to the discrepancy stop for every scene (batched GPU solves).
    Returns (g, f, b, iterations) as CUDA tensors / numpy."""
    import torch
    Hs = scs[0].g.shape[1]
    g_all = torch.empty((len(scs), Hs, Hs), dtype=torch.float32, device="cuda")
    f_all = torch.empty_like(g_all)
    b_all = torch.tensor([float(s.b[0]) for s in scs], dtype=torch.float32, device="cuda")
    its = np.zeros(len(scs), np.int64)
    for a in range(0, len(scs), batch):
        part = scs[a:a + batch]
        probs = lib.Problems([torch.from_numpy(s.psfs.astype(np.float32)).cuda() for s in part],
                             [[float(s.b[0])] for s in part])
        for i, s in enumerate(part):
            g = torch.from_numpy(s.g.astype(np.float32)).cuda()
            probs.set_data(i, g)
            g_all[a + i].copy_(g[0])
        it = probs.solve_until(lib.STOP_DISCREPANCY, max_iter=max_iter, eta=1.0, raise_on_error=False)
        for i in range(len(part)):
            probs.get_f(i, out=f_all[a + i])
        its[a:a + len(part)] = it
        probs.close()
    return g_all, f_all, b_all, its


def train(net: WarmStartNet, g, f, b, epochs: int = 3, batch: int = 32, lr: float = 2e-3, seed: int = 0,
          log=None) -> list[float]:
    """Adam on the squared error of the log-domain correction; batches are contiguous slices of the
    (pre-shuffled) data visited in a random order each epoch."""
    import torch
    n, H, W = g.shape
    rng = np.random.default_rng(seed)
    nb = n // batch
    losses = []
    for ep in range(epochs):
        tot = torch.zeros(1, dtype=torch.float64, device="cuda")
        for k in rng.permutation(nb):
            sl = slice(k * batch, (k + 1) * batch)
            bf = net.prepare(g[sl], b[sl], f[sl])
            net.loss_and_grad(bf, batch, H, W)
            net.adam(lr * (0.5 ** ep))
            tot += bf["loss"]
        losses.append(float(tot.item()) / (nb * batch * H * W))
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.4e}")
    return losses


def train_crops(net: WarmStartNet, g, f, b, steps: int = 200, crop: int = 512, batch: int = 8, lr: float = 2e-3,
                seed: int = 0) -> list[float]:
    """Adam on random crop x crop windows of (g, f) pairs of larger images (B, H, W CUDA tensors):
    the network is local (3 x 3 convolutions, one 2 x 2 pooling level), so windows of the images
    teach it the same mapping at a fraction of the cost of whole images.  lr halves at 1/2 and 3/4
    of the steps.  Returns the loss of each step."""
    import torch
    n, H, W = g.shape
    rng = np.random.default_rng(seed)
    losses = []
    gb = torch.empty((batch, crop, crop), dtype=torch.float32, device=g.device)
    fb = torch.empty_like(gb)
    bb = torch.empty(batch, dtype=torch.float32, device=g.device)
    for step in range(steps):
        for k in range(batch):
            i = int(rng.integers(n))
            y0, x0 = int(rng.integers(0, H - crop + 1)), int(rng.integers(0, W - crop + 1))
            gb[k].copy_(g[i, y0:y0 + crop, x0:x0 + crop])
            fb[k].copy_(f[i, y0:y0 + crop, x0:x0 + crop])
            bb[k] = b[i]
        bf = net.prepare(gb, bb, fb)
        net.loss_and_grad(bf, batch, crop, crop)
        net.adam(lr * (0.5 if step >= steps // 2 else 1.0) * (0.5 if step >= 3 * steps // 4 else 1.0))
        losses.append(bf["loss"].clone())
    return [float(x.item()) / (batch * crop * crop) for x in losses]


LAND_TOL = 1e-5   # both starts end with the discrepancy in [1 - LAND_TOL, 1]: equal final KL


def evaluate(net: WarmStartNet, scs, max_iter: int = 2000, batch: int = 50, n_single: int = 100):
    """Flat-start vs warm-start SGP to the same landed discrepancy stop (the last step shortened so
    that the discrepancy ends in [1 - LAND_TOL, 1]): iterations, GPU time, final KL.

    Batched: every image of a batch of `batch` problems gets its own stop, the batch time is the time
    until all have stopped.  Single: the first `n_single` images solved one at a time, each solve
    timed after a first untimed solve has built the context's graph (flat: constant start; warm:
    network forward + solve from its f^(0))."""
    import torch
    out = {"flat_iters": [], "warm_iters": [], "flat_kl": [], "warm_kl": [], "flat_ms": 0.0, "warm_ms": 0.0,
           "net_ms": 0.0, "fallbacks": 0, "single_flat_ms": [], "single_warm_ms": [], "single_net_ms": [],
           "single_flat32_ms": [], "single_kl_rel_warm_flat32": [], "single_failed": {}, "net_errors": 0}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for a in range(0, len(scs), batch):
        part = scs[a:a + batch]
        psf = [torch.from_numpy(s.psfs.astype(np.float32)).cuda() for s in part]
        bc = [[float(s.b[0])] for s in part]
        g = torch.stack([torch.from_numpy(s.g[0].astype(np.float32)) for s in part]).cuda()
        bvec = torch.tensor([float(s.b[0]) for s in part], dtype=torch.float32, device="cuda")
        for mode in ("flat", "warm"):
            probs = lib.Problems(psf, bc)
            for i in range(len(part)):
                probs.set_data(i, g[i:i + 1])
            torch.cuda.synchronize()
            ev[0].record()
            if mode == "warm":
                f0 = net.predict(g, bvec)
                ev[2].record()
                for i in range(len(part)):
                    probs.set_start(i, lib.START_USER, f0[i])
                out["net_errors"] += device_error()
            it = probs.solve_until(lib.STOP_LANDED, max_iter=max_iter, eta=1.0, tol=LAND_TOL, raise_on_error=False)
            ev[1].record()
            torch.cuda.synchronize()
            out[f"{mode}_ms"] += ev[0].elapsed_time(ev[1])
            if mode == "warm":
                out["net_ms"] += ev[0].elapsed_time(ev[2])
            infos = [probs.info(i) for i in range(len(part))]
            if mode == "warm":
                # a start the method cannot use falls back to the flat start (its flat result stands)
                bad = [i for i, inf in enumerate(infos) if inf.status != 0]
                out["fallbacks"] += len(bad)
                base = len(out["warm_iters"])
                it = list(it)
                for i in bad:
                    it[i] = out["flat_iters"][base + i]
                klw = [inf.J if inf.status == 0 else out["flat_kl"][base + i] for i, inf in enumerate(infos)]
            else:
                klw = [inf.J for inf in infos]
            out[f"{mode}_iters"] += list(it)
            out[f"{mode}_kl"] += klw
            probs.close()
    for sc in scs[:n_single]:
        psf = torch.from_numpy(sc.psfs.astype(np.float32)).cuda()
        g = torch.from_numpy(sc.g.astype(np.float32)).cuda()
        bvec = torch.tensor([float(sc.b[0])], dtype=torch.float32, device="cuda")
        prob = lib.Problems(psf, [float(sc.b[0])])
        prob.set_data(0, g)
        f0 = net.predict(g, bvec)
        prob.solve_until(lib.STOP_LANDED, max_iter=max_iter, eta=1.0, tol=LAND_TOL, raise_on_error=False)   # graph
        # the plain FP32 single-image form (FP32 reductions and decisions, flat start)
        prob32 = lib.Problems(psf, [float(sc.b[0])], params=lib.default_params(reduce_fp64=0))
        prob32.set_data(0, g)
        prob32.solve_until(lib.STOP_LANDED, max_iter=max_iter, eta=1.0, tol=LAND_TOL, raise_on_error=False)
        times, kls = {}, {}
        for mode in ("flat", "warm", "flat32"):
            pr = prob32 if mode == "flat32" else prob
            torch.cuda.synchronize()
            ev[0].record()
            if mode == "warm":
                f0 = net.predict(g, bvec)
                ev[2].record()
                pr.set_start(0, lib.START_USER, f0[0])
            else:
                pr.set_start(0, lib.START_CONSTANT)
            pr.solve_until(lib.STOP_LANDED, max_iter=max_iter, eta=1.0, tol=LAND_TOL, raise_on_error=False)
            ev[1].record()
            torch.cuda.synchronize()
            inf = pr.info(0)
            times[mode] = ev[0].elapsed_time(ev[1]) if inf.status == 0 and inf.stopped else None
            if inf.status != 0:   # record the failure (status code per arm); the image is left out
                key = f"{mode}:{lib.STATUS_NAMES[inf.status]}"
                out["single_failed"][key] = out["single_failed"].get(key, 0) + 1
            kls[mode] = pr.get_f(0).clone() if inf.status == 0 else None
            if mode == "warm":
                times["net"] = ev[0].elapsed_time(ev[2])
                out["net_errors"] += device_error()
        # final KL of the warm (mixed) and plain-FP32 results, both evaluated with FP64 accumulation
        for mode in ("warm", "flat32"):
            if kls[mode] is None:
                continue
            try:
                prob.set_start(0, lib.START_USER, kls[mode])
                kls[mode] = prob.kl_value(0)
            except lib.SGPError as e:
                key = f"{mode}:kl_eval:{lib.STATUS_NAMES[e.status]}"
                out["single_failed"][key] = out["single_failed"].get(key, 0) + 1
                kls[mode] = None
        if kls["warm"] is None or kls["flat32"] is None:
            prob.close()
            prob32.close()
            continue
        if times["flat"] is not None and times["warm"] is not None:
            out["single_flat_ms"].append(times["flat"])
            out["single_warm_ms"].append(times["warm"])
            out["single_net_ms"].append(times["net"])
            if times["flat32"] is not None:
                out["single_flat32_ms"].append(times["flat32"])
                out["single_kl_rel_warm_flat32"].append(abs(kls["warm"] - kls["flat32"]) / kls["flat32"])
        prob.close()
        prob32.close()
    for k in ("flat_iters", "warm_iters", "flat_kl", "warm_kl", "single_flat_ms", "single_warm_ms", "single_net_ms",
              "single_flat32_ms", "single_kl_rel_warm_flat32"):
        out[k] = np.asarray(out[k])
    return out


def _scene_chunk(args):
    n, N, seed = args
    sc = make_scenes(n, N, seed)
    return [(s.psfs.astype(np.float32), s.g.astype(np.float32), float(s.b[0])) for s in sc]


def _light(items):
    out = []
    for psf, g, b in items:
        out.append(scenes.Scene(psfs=psf, g=g, b=np.array([b]), f_true=None))
    return out


def generate(n: int, N: int, seed: int, workers: int = 0):
    """n seeded scenes of side N, generated in parallel worker processes (spawned, before any GPU
    work in them)."""
    import multiprocessing as mp
    import os
    workers = workers or min(16, os.cpu_count() or 1)
    chunk = max(1, n // (4 * workers))
    jobs = [(min(chunk, n - a), N, seed * 100003 + a) for a in range(0, n, chunk)]
    if workers <= 1:
        res = [_scene_chunk(j) for j in jobs]
    else:
        with mp.get_context("spawn").Pool(workers) as pool:
            res = pool.map(_scene_chunk, jobs)
    return _light([x for r in res for x in r])


def main(argv=None) -> int:
    """Train the warm start on SGP solutions and compare warm vs flat starts on held-out images.

    python -m paper_1210_2258_b300.warmstart --train 20000 --train-side 256 --eval 1000 --eval-side 512
    """
    import argparse
    import json
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=20000)
    ap.add_argument("--train-side", type=int, default=256)
    ap.add_argument("--eval", type=int, default=1000)
    ap.add_argument("--eval-side", type=int, default=512)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--max-iter", type=int, default=400)
    ap.add_argument("--save", default="")
    a = ap.parse_args(argv)
    log = lambda m: print(m, flush=True)
    t0 = time.perf_counter()
    tr = generate(a.train, a.train_side, seed=1)
    ev_scenes = generate(a.eval, a.eval_side, seed=2)
    t1 = time.perf_counter()
    log(f"scenes: {len(tr)} train {a.train_side}^2, {len(ev_scenes)} eval {a.eval_side}^2 in {t1 - t0:.1f} s")
    torch.cuda.synchronize()
    g, f, b, its = sgp_solutions(tr, max_iter=a.max_iter)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    log(f"training targets: {len(tr)} SGP solves in {t2 - t1:.1f} s, mean iterations {its.mean():.1f}, "
        f"stopped {np.mean(its < a.max_iter) * 100:.1f}%")
    net = WarmStartNet(seed=0)
    losses = train(net, g, f, b, epochs=a.epochs, batch=a.batch, lr=a.lr, log=log)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    res = evaluate(net, ev_scenes)
    t4 = time.perf_counter()
    done = (res["flat_iters"] < 2000) & (res["warm_iters"] < 2000)
    single = {}
    if len(res["single_flat_ms"]):
        single = {"single_images": int(len(res["single_flat_ms"])),
                  "single_flat_ms_median": float(np.median(res["single_flat_ms"])),
                  "single_warm_ms_median": float(np.median(res["single_warm_ms"])),
                  "single_net_ms_median": float(np.median(res["single_net_ms"])),
                  "single_warm_faster_frac": float(np.mean(res["single_warm_ms"] < res["single_flat_ms"]))}
        if len(res["single_flat32_ms"]) == len(res["single_warm_ms"]):
            single.update({"single_flat_plain_fp32_ms_median": float(np.median(res["single_flat32_ms"])),
                           "single_warm_faster_than_plain_fp32_frac":
                               float(np.mean(res["single_warm_ms"] < res["single_flat32_ms"])),
                           "single_kl_rel_warm_vs_plain_fp32_max": float(np.max(res["single_kl_rel_warm_flat32"])),
                           "single_kl_rel_warm_vs_plain_fp32_median":
                               float(np.median(res["single_kl_rel_warm_flat32"])),
                           "single_kl_rel_warm_vs_plain_fp32_le_1e-4_frac":
                               float(np.mean(res["single_kl_rel_warm_flat32"] <= 1e-4))})
    kl_rel = np.abs(res["warm_kl"] - res["flat_kl"]) / res["flat_kl"]
    summary = {
        "train_pairs": len(tr), "train_side": a.train_side, "eval_images": len(ev_scenes), "eval_side": a.eval_side,
        "target_solves_s": t2 - t1, "target_mean_iters": float(its.mean()), "train_s": t3 - t2,
        "train_loss_first_last": [losses[0], losses[-1]],
        "both_stopped": int(done.sum()),
        "flat_mean_iters": float(res["flat_iters"][done].mean()), "warm_mean_iters": float(res["warm_iters"][done].mean()),
        "flat_gpu_ms_total": res["flat_ms"], "warm_gpu_ms_total": res["warm_ms"], "net_ms_total": res["net_ms"],
        "final_kl_rel_diff_median": float(np.median(kl_rel[done])), "final_kl_rel_diff_max": float(np.max(kl_rel[done])),
        "flat_not_stopped": int((res["flat_iters"] >= 2000).sum()),
        "warm_not_stopped": int((res["warm_iters"] >= 2000).sum()),
        "eval_s": t4 - t3, "fallbacks_to_flat": res["fallbacks"], "single_failed": res["single_failed"],
        "net_device_errors": res["net_errors"], **single,
    }
    log(json.dumps(summary))
    if a.save:
        np.savez(a.save, **net.params())
    return 0


if __name__ == "__main__":
    import sys
    sys.exit(main())
