"""ctypes binding of the native deconvolution library (include/sgp.h).

Argument marshalling only: every step of RL and SGP runs in the library's CUDA kernels.  PyTorch
provides device memory (the workspace and the arrays handed to the library) and streams.  There
is no CPU fallback: load() raises if the native library is missing.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("SGP_LIB_PATH") or os.path.join(HERE, "lib", "libsgp_b300.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "sgp.h")

OK, ERR_ARG, ERR_SIZE, ERR_PSF, ERR_CUDA, ERR_WORKSPACE, ERR_LINESEARCH, ERR_TIMEOUT, ERR_NONFINITE, ERR_STATE = range(10)
STATUS_NAMES = ["OK", "ARG", "SIZE_UNSUPPORTED", "PSF", "CUDA", "WORKSPACE", "LINESEARCH", "TIMEOUT",
                "NONFINITE", "STATE"]
STOP_FIXED, STOP_CONVERGENCE, STOP_DISCREPANCY, STOP_MIN_ERROR, STOP_LANDED = range(5)
START_ZERO, START_DATA, START_CONSTANT, START_USER = range(4)
PSF_CENTER, PSF_CORNER = 0, 1
N_PASSES = 7    # passes of one SGP iteration (sgp_time_passes)
MAX_VIEWS = 8   # views per problem (sgp_inputs.b_const)
SIDES = (16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048)


class Shape(C.Structure):
    _fields_ = [("H", C.c_int), ("W", C.c_int), ("p", C.c_int), ("has_mask", C.c_int), ("psf_origin", C.c_int)]


class Params(C.Structure):
    _fields_ = [("beta", C.c_double), ("theta", C.c_double), ("alpha0", C.c_double), ("tau1", C.c_double),
                ("alpha_min", C.c_double), ("alpha_max", C.c_double), ("M_alpha", C.c_int),
                ("warmup_iters", C.c_int), ("adaptive_L", C.c_int), ("max_backtracks", C.c_int),
                ("L1", C.c_double), ("L2", C.c_double), ("sigma_R", C.c_double), ("constraint", C.c_int),
                ("flux_c", C.c_double), ("reduce_fp64", C.c_int), ("trace_cap", C.c_int),
                ("band_tol", C.c_double), ("reg_beta", C.c_double)]


class StopRule(C.Structure):
    _fields_ = [("kind", C.c_int), ("max_iter", C.c_int), ("tol", C.c_double), ("eta", C.c_double)]


class Inputs(C.Structure):
    _fields_ = [("psfs", C.c_void_p), ("b", C.c_void_p), ("b_const", C.c_float * 8), ("mask", C.c_void_p)]


class Info(C.Structure):
    _fields_ = [("k", C.c_int), ("status", C.c_int), ("stopped", C.c_int), ("trace_n", C.c_int),
                ("J", C.c_double), ("D", C.c_double), ("L1", C.c_double), ("L2", C.c_double),
                ("alpha", C.c_double), ("tau", C.c_double), ("lambda_", C.c_double), ("rho", C.c_double),
                ("nS", C.c_double), ("flux_c", C.c_double), ("band_cols", C.c_int), ("reg", C.c_double)]


class Mosaic(C.Structure):
    _fields_ = [("H", C.c_int), ("W", C.c_int), ("ny", C.c_int), ("nx", C.c_int), ("sub_h", C.c_int),
                ("sub_w", C.c_int), ("ext_h", C.c_int), ("ext_w", C.c_int)]


_lib = None


def load() -> C.CDLL:
    """Load the native library (built in-tree by build.py); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"native library not built: {LIB_PATH} (run python -m paper_1210_2258_b300.build)")
    lib = C.CDLL(LIB_PATH)
    vp, i, d, st = C.c_void_p, C.c_int, C.c_double, C.c_int
    sig = {
        "sgp_params_default": (None, [C.POINTER(Params)]),
        "sgp_workspace_bytes": (C.c_size_t, [i, C.POINTER(Shape), C.POINTER(Params)]),
        "sgp_create_batch": (st, [C.POINTER(vp), i, C.POINTER(Shape), C.POINTER(Inputs), C.POINTER(Params), vp,
                                  C.c_size_t, vp]),
        "sgp_create": (st, [C.POINTER(vp), C.POINTER(Shape), vp, vp, C.POINTER(C.c_float), vp,
                            C.POINTER(Params), vp, C.c_size_t, vp]),
        "sgp_set_data": (st, [vp, i, vp]),
        "sgp_set_start": (st, [vp, i, i, vp]),
        "sgp_set_truth": (st, [vp, i, vp]),
        "rl_iterate": (st, [vp, i]),
        "sgp_iterate": (st, [vp, i]),
        "osem_iterate": (st, [vp, i]),
        "sgp_solve_until": (st, [vp, C.POINTER(StopRule), C.POINTER(C.c_int)]),
        "rl_solve_until": (st, [vp, C.POINTER(StopRule), C.POINTER(C.c_int)]),
        "kl_value": (st, [vp, i, C.POINTER(d)]),
        "sgp_get_f": (st, [vp, i, vp]),
        "sgp_get_trace": (st, [vp, i, C.POINTER(d), i, C.POINTER(C.c_int)]),
        "sgp_get_info": (st, [vp, i, C.POINTER(Info)]),
        "sgp_apply_A": (st, [vp, i, vp, vp]),
        "sgp_apply_AT": (st, [vp, i, vp, vp]),
        "sgp_time_passes": (st, [vp, i, C.POINTER(d), i]),
        "sgp_launch_count": (C.c_longlong, [vp]),
        "sgp_get_tile": (st, [vp, C.POINTER(i), C.POINTER(i)]),
        "sgp_set_tile": (st, [vp, i]),
        "sgp_convolve_noalloc": (st, [vp, vp, vp, i, i, i, i, vp]),
        "sgp_mosaic_geometry": (st, [C.POINTER(Mosaic), C.POINTER(i)]),
        "sgp_mosaic_split": (st, [C.POINTER(Mosaic), i, vp, vp, vp, vp]),
        "sgp_mosaic_stitch": (st, [C.POINTER(Mosaic), vp, vp, vp]),
        "sgp_sum_terms_workspace_bytes": (C.c_size_t, [C.c_size_t]),
        "sgp_sum_terms": (st, [i, i, vp, vp, vp, C.c_size_t, d, vp, C.POINTER(d), vp, C.c_size_t, vp]),
        "sgp_destroy": (st, [vp]),
        "sgp_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def header_symbols() -> list[str]:
    """Names of the entry points declared in include/sgp.h and include/warmstart.h."""
    names = []
    for h, tag in ((HEADER, "SGP_API"), (os.path.join(os.path.dirname(HEADER), "warmstart.h"), "WS_API")):
        txt = open(h).read()
        names += re.findall(tag + r"\s+[\w\s\*]+?\b(\w+)\s*\(", txt)
    return names


class SGPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"SGP_ERR_{name}: {msg}")


def _check(status: int) -> None:
    if status != OK:
        raise SGPError(status, load().sgp_last_error().decode())


def default_params(**kw) -> Params:
    p = Params()
    load().sgp_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _stream_ptr(stream) -> int | None:
    return None if stream is None else stream.cuda_stream


class Problems:
    """A context of n problems (same H, W, p) advancing together on one GPU.

    psfs: list of (p, H, W) float32 CUDA tensors (or one tensor for n = 1); b: list of p-tuples
    of constant backgrounds (or (p, H, W) CUDA tensors); masks: list of (H, W) uint8 CUDA
    tensors (boundary problems) or None.  The workspace is a torch uint8 tensor owned here."""

    def __init__(self, psfs, b, masks=None, params: Params | None = None, psf_origin: int = PSF_CENTER,
                 stream=None):
        import torch
        lib = load()
        if not isinstance(psfs, (list, tuple)):
            psfs, b, masks = [psfs], [b], [masks]
        n = len(psfs)
        masks = masks if masks is not None else [None] * n
        self.n = n
        self.p, self.H, self.W = (int(s) for s in psfs[0].shape)
        if self.p > MAX_VIEWS:
            raise SGPError(ERR_ARG, f"at most {MAX_VIEWS} views per problem")
        self.params = params or default_params()
        shapes = (Shape * n)()
        inputs = (Inputs * n)()
        self._keep = []
        self.shapes = [tuple(int(v) for v in ps.shape[-2:]) for ps in psfs]
        for k in range(n):
            ps = psfs[k].contiguous()
            self._keep.append(ps)
            Hk, Wk = self.shapes[k]
            shapes[k] = Shape(Hk, Wk, self.p, 1 if masks[k] is not None else 0, psf_origin)
            inputs[k].psfs = ps.data_ptr()
            bk = b[k]
            if hasattr(bk, "data_ptr"):
                bk = bk.contiguous()
                self._keep.append(bk)
                inputs[k].b = bk.data_ptr()
            else:
                vals = list(np.broadcast_to(np.asarray(bk, np.float32), (self.p,)))
                for j in range(self.p):
                    inputs[k].b_const[j] = float(vals[j])
            if masks[k] is not None:
                m = masks[k].to(torch.uint8).contiguous()
                self._keep.append(m)
                inputs[k].mask = m.data_ptr()
        nbytes = lib.sgp_workspace_bytes(n, shapes, C.byref(self.params))
        if nbytes == 0:
            _check(ERR_SIZE)
        self.device = psfs[0].device
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        self.ctx = C.c_void_p()
        self.stream = stream
        _check(lib.sgp_create_batch(C.byref(self.ctx), n, shapes, inputs, C.byref(self.params),
                                    C.c_void_p(aligned), C.c_size_t(nbytes), _stream_ptr(stream)))
        self._keep = []

    # ------------------------------------------------------------------ data and state
    def set_data(self, image: int, g) -> None:
        g = g.contiguous()
        _check(load().sgp_set_data(self.ctx, image, g.data_ptr()))

    def set_start(self, image: int, mode: int, f0=None) -> None:
        f0c = f0.contiguous() if f0 is not None else None
        _check(load().sgp_set_start(self.ctx, image, mode, _ptr(f0c)))
        # the call is stream-ordered: a contiguous copy made here stays alive until the next start
        # of this image, so that its memory is not reused before the library has read it
        self._starts = getattr(self, "_starts", {})
        self._starts[image] = f0c

    def set_truth(self, image: int, f_true) -> None:
        self._truth = getattr(self, "_truth", {})
        self._truth[image] = f_true.contiguous() if f_true is not None else None
        _check(load().sgp_set_truth(self.ctx, image, _ptr(self._truth[image])))

    # ------------------------------------------------------------------ iterations
    def rl_iterate(self, n: int) -> None:
        _check(load().rl_iterate(self.ctx, n))

    def sgp_iterate(self, n: int) -> None:
        _check(load().sgp_iterate(self.ctx, n))

    def osem_iterate(self, n: int) -> None:
        """n OSEM iterations (Algorithm 2; boundary form with a mask)."""
        _check(load().osem_iterate(self.ctx, n))

    def solve_until(self, kind: int, max_iter: int = 100000, tol: float = 0.0, eta: float = 1.0,
                    method: str = "sgp", raise_on_error: bool = True) -> list[int]:
        rule = StopRule(kind, max_iter, tol, eta)
        iters = (C.c_int * self.n)()
        fn = load().sgp_solve_until if method == "sgp" else load().rl_solve_until
        st = fn(self.ctx, C.byref(rule), iters)
        if raise_on_error:
            _check(st)
        self.last_status = st
        return list(iters)

    # ------------------------------------------------------------------ results
    def kl_value(self, image: int = 0) -> float:
        out = C.c_double()
        _check(load().kl_value(self.ctx, image, C.byref(out)))
        return out.value

    def info(self, image: int = 0) -> Info:
        out = Info()
        _check(load().sgp_get_info(self.ctx, image, C.byref(out)))
        return out

    def get_f(self, image: int = 0, out=None):
        import torch
        if out is None:
            out = torch.empty(self.shapes[image], dtype=torch.float32, device=self.device)
        _check(load().sgp_get_f(self.ctx, image, out.data_ptr()))
        return out

    def trace(self, image: int = 0) -> np.ndarray:
        cnt = C.c_int()
        _check(load().sgp_get_trace(self.ctx, image, None, 0, C.byref(cnt)))
        buf = (C.c_double * (8 * max(cnt.value, 1)))()
        _check(load().sgp_get_trace(self.ctx, image, buf, cnt.value, C.byref(cnt)))
        return np.frombuffer(buf, dtype=np.float64).reshape(-1, 8)[:cnt.value].copy()

    # ------------------------------------------------------------------ operators
    def apply_A(self, f, image: int = 0, out=None):
        import torch
        f = f.contiguous()
        if out is None:
            out = torch.empty((self.p,) + self.shapes[image], dtype=torch.float32, device=self.device)
        _check(load().sgp_apply_A(self.ctx, image, f.data_ptr(), out.data_ptr()))
        return out

    def apply_AT(self, y, image: int = 0, out=None):
        import torch
        y = y.contiguous()
        if out is None:
            out = torch.empty(self.shapes[image], dtype=torch.float32, device=self.device)
        _check(load().sgp_apply_AT(self.ctx, image, y.data_ptr(), out.data_ptr()))
        return out

    def time_passes(self, iters: int = 5) -> list[float]:
        """Mean duration (ms) of each of the 7 passes of an SGP iteration (CUDA events)."""
        out = (C.c_double * N_PASSES)()
        _check(load().sgp_time_passes(self.ctx, iters, out, N_PASSES))
        return list(out)

    def launch_count(self) -> int:
        return int(load().sgp_launch_count(self.ctx))

    def tile(self) -> tuple[int, int]:
        """(rows per work item, threads per block) of the hot row passes."""
        r, t = C.c_int(), C.c_int()
        _check(load().sgp_get_tile(self.ctx, C.byref(r), C.byref(t)))
        return r.value, t.value

    def set_tile(self, rows: int) -> None:
        _check(load().sgp_set_tile(self.ctx, rows))

    def close(self) -> None:
        if getattr(self, "ctx", None):
            load().sgp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


SUM_VALUES, SUM_KL, SUM_ARMIJO, SUM_BB0 = 0, 1, 2, 3


def sum_terms(kind: int, a, b=None, c=None, lam: float = 1.0, reduce_fp64: int = 1, want_terms: bool = True,
              stream=None):
    """Pixel terms of one kind and their sum through the library's reduction (sgp_sum_terms).
    a, b, c: float32 CUDA tensors of equal size.  Returns (sum as float, terms tensor or None)."""
    import torch
    lib = load()
    n = a.numel()
    ws = torch.empty(lib.sgp_sum_terms_workspace_bytes(n) + 256, dtype=torch.uint8, device=a.device)
    base = (ws.data_ptr() + 255) & ~255
    terms = torch.empty_like(a) if want_terms else None
    out = C.c_double()
    _check(lib.sgp_sum_terms(kind, reduce_fp64, a.data_ptr(), _ptr(b), _ptr(c), n, lam, _ptr(terms),
                             C.byref(out), C.c_void_p(base), ws.numel() - (base - ws.data_ptr()),
                             _stream_ptr(stream)))
    return out.value, terms


def single(psf, g, b, mask=None, params: Params | None = None, stream=None) -> Problems:
    """One problem from torch CUDA tensors psf (p,H,W) or (H,W), g likewise; b constants or tensor."""
    if psf.dim() == 2:
        psf, g = psf[None], g[None]
    prob = Problems(psf, b if hasattr(b, "data_ptr") else np.atleast_1d(b), mask, params, stream=stream)
    prob.set_data(0, g)
    return prob
