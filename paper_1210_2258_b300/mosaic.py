"""Mosaic of boundary-corrected reconstructions (Sect. 4, second experiment; Table 2, Table 6).

An H x W image is covered by ny x nx partially overlapping sub-domains; every sub-image is merged
by zero padding into an extended array (the sub-image centred, mask M_S = 1 on it), all of them
are reconstructed together in one context of boundary problems (one set of launches per pass),
and the mosaic keeps a non-overlapping piece of each reconstruction.  Splitting and stitching
run in the library's kernels (sgp_mosaic_split / sgp_mosaic_stitch); this module only marshals.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import sgp as lib


def geometry(H: int, W: int, n=(2, 2), sub=(160, 160), ext=(256, 256)):
    """(sub-domain start, end, piece start, end) per sub-domain along H, then along W."""
    m = lib.Mosaic(H, W, n[0], n[1], sub[0], sub[1], ext[0], ext[1])
    out = (C.c_int * (4 * (n[0] + n[1])))()
    lib._check(lib.load().sgp_mosaic_geometry(C.byref(m), out))
    v = list(out)
    q = [tuple(v[4 * k:4 * k + 4]) for k in range(n[0] + n[1])]
    return q[:n[0]], q[n[0]:]


class MosaicSolver:
    """g: (p, H, W) CUDA float32 data; psfs_ext: (p, EH, EW) CUDA float32 PSFs on the extended
    array (centred); b: p constant backgrounds.  The tiles' context is created once; solve()
    can be called again after set_data()."""

    def __init__(self, psfs_ext, g, b, n=(2, 2), sub=(160, 160), ext=(256, 256), params=None, stream=None):
        import torch
        if g.dim() == 2:
            g = g[None]
        self.p, self.H, self.W = (int(v) for v in g.shape)
        self.n, self.sub, self.ext = tuple(n), tuple(sub), tuple(ext)
        self.m = lib.Mosaic(self.H, self.W, n[0], n[1], sub[0], sub[1], ext[0], ext[1])
        self.nt = n[0] * n[1]
        self.stream = stream
        dev = g.device
        self.tiles = torch.empty((self.nt, self.p) + self.ext, dtype=torch.float32, device=dev)
        self.masks = torch.empty((self.nt,) + self.ext, dtype=torch.uint8, device=dev)
        self.recs = torch.empty((self.nt,) + self.ext, dtype=torch.float32, device=dev)
        self._split(g)
        psfs_ext = psfs_ext if psfs_ext.dim() == 3 else psfs_ext[None]
        bl = list(np.broadcast_to(np.asarray(b, np.float32), (self.p,)))
        self.prob = lib.Problems([psfs_ext] * self.nt, [bl] * self.nt, [self.masks[t] for t in range(self.nt)],
                                 params, stream=stream)
        for t in range(self.nt):
            self.prob.set_data(t, self.tiles[t])

    def _split(self, g):
        g = g.contiguous()
        lib._check(lib.load().sgp_mosaic_split(C.byref(self.m), self.p, g.data_ptr(), self.tiles.data_ptr(),
                                               self.masks.data_ptr(), lib._stream_ptr(self.stream)))

    def set_data(self, g) -> None:
        """New data of the same geometry (the masks do not change)."""
        self._split(g if g.dim() == 3 else g[None])
        for t in range(self.nt):
            self.prob.set_data(t, self.tiles[t])

    def solve(self, method: str = "sgp", n_iter: int | None = 50, stop: int | None = None, max_iter: int = 3000,
              eta: float = 1.0, out=None):
        """n_iter iterations of SGP / RL / OSEM on every tile (or, with stop, SGP/RL to that rule),
        then the mosaic (H, W)."""
        import torch
        for t in range(self.nt):
            self.prob.set_start(t, lib.START_CONSTANT)
        if stop is not None:
            self.iters = self.prob.solve_until(stop, max_iter=max_iter, eta=eta, method=method, raise_on_error=False)
        elif method == "sgp":
            self.prob.sgp_iterate(n_iter)
        elif method == "rl":
            self.prob.rl_iterate(n_iter)
        else:
            self.prob.osem_iterate(n_iter)
        for t in range(self.nt):
            self.prob.get_f(t, out=self.recs[t])
        if out is None:
            out = torch.empty((self.H, self.W), dtype=torch.float32, device=self.recs.device)
        lib._check(lib.load().sgp_mosaic_stitch(C.byref(self.m), self.recs.data_ptr(), out.data_ptr(),
                                                lib._stream_ptr(self.stream)))
        return out
