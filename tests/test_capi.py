"""The native library loads, exports every entry point declared in include/sgp.h, and its host-side
validation rejects bad arguments before touching a GPU (CPU only)."""
import ctypes as C
import os

import pytest

from paper_1210_2258_b300 import sgp as S


def test_library_exports_every_declared_symbol():
    lib = S.load()
    names = S.header_symbols()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n


def test_default_parameters_are_the_papers():
    p = S.default_params()
    assert (p.beta, p.theta, p.alpha0, p.tau1, p.alpha_min, p.alpha_max) == (1e-4, 0.4, 1.3, 0.5, 1e-5, 1e5)
    assert (p.M_alpha, p.warmup_iters, p.adaptive_L, p.reduce_fp64) == (3, 20, 1, 1)


def test_workspace_bytes_and_size_validation():
    lib = S.load()
    sh = (S.Shape * 1)(S.Shape(256, 256, 1, 0, 0))
    small = lib.sgp_workspace_bytes(1, sh, None)
    sh3 = (S.Shape * 1)(S.Shape(256, 256, 3, 0, 0))
    assert lib.sgp_workspace_bytes(1, sh3, None) > small > 10 * 256 * 256 * 4
    for bad in [(100, 256, 1), (256, 4096, 1), (256, 256, 0), (256, 256, 9), (8, 16, 1)]:
        shb = (S.Shape * 1)(S.Shape(bad[0], bad[1], bad[2], 0, 0))
        assert lib.sgp_workspace_bytes(1, shb, None) == 0


def test_create_rejects_bad_arguments_without_gpu_work():
    lib = S.load()
    ctx = C.c_void_p()
    sh = S.Shape(100, 256, 1, 0, 0)
    st = lib.sgp_create(C.byref(ctx), C.byref(sh), None, None, None, None, None, None, 0, None)
    assert st == S.ERR_SIZE and b"power of two" in lib.sgp_last_error()
    sh = S.Shape(256, 256, 1, 1, 0)   # mask requested but not given
    st = lib.sgp_create(C.byref(ctx), C.byref(sh), C.c_void_p(256), None, (C.c_float * 1)(1.0), None,
                        None, C.c_void_p(256), 1 << 30, None)
    assert st == S.ERR_ARG
    assert lib.rl_iterate(None, 1) == S.ERR_ARG


def test_regularisation_weight_is_validated_before_gpu_work():
    lib = S.load()
    ctx = C.c_void_p()
    sh = S.Shape(256, 256, 1, 0, 0)
    for bad in (-1e-3, float("nan"), float("inf")):
        p = S.default_params(reg_beta=bad)
        st = lib.sgp_create(C.byref(ctx), C.byref(sh), C.c_void_p(256), None, (C.c_float * 1)(1.0), None,
                            C.byref(p), C.c_void_p(256), 1 << 30, None)
        assert st == S.ERR_ARG and b"reg_beta" in lib.sgp_last_error(), bad
    assert S.default_params().reg_beta == 0.0


def test_sum_terms_rejects_bad_arguments_without_gpu_work():
    """sgp_sum_terms checks its arguments and workspace before any CUDA call (pointers here are
    never dereferenced)."""
    lib = S.load()
    n = 1 << 20
    need = lib.sgp_sum_terms_workspace_bytes(n)
    assert need >= 2048 and lib.sgp_sum_terms_workspace_bytes(4 * n) > need
    assert lib.sgp_sum_terms_workspace_bytes(1) >= 2048
    a, b, c, w = C.c_void_p(256), C.c_void_p(512), C.c_void_p(768), C.c_void_p(1 << 20)
    out = C.c_double()
    call = lambda kind, a, b, c, n, outp, ws, wsb: lib.sgp_sum_terms(kind, 1, a, b, c, n, 1.0, None, outp, ws,
                                                                     wsb, None)
    assert call(S.SUM_VALUES, a, None, None, n, None, w, need) == S.ERR_ARG
    assert call(S.SUM_VALUES, None, None, None, n, C.byref(out), w, need) == S.ERR_ARG
    assert call(S.SUM_VALUES, a, None, None, 0, C.byref(out), w, need) == S.ERR_ARG
    assert call(99, a, b, c, n, C.byref(out), w, need) == S.ERR_ARG
    assert call(-1, a, b, c, n, C.byref(out), w, need) == S.ERR_ARG
    assert call(S.SUM_KL, a, None, None, n, C.byref(out), w, need) == S.ERR_ARG
    assert call(S.SUM_ARMIJO, a, b, None, n, C.byref(out), w, need) == S.ERR_ARG
    assert call(S.SUM_BB0 + 3, a, b, None, n, C.byref(out), w, need) == S.ERR_ARG
    assert call(S.SUM_VALUES, a, None, None, n, C.byref(out), None, need) == S.ERR_WORKSPACE
    assert call(S.SUM_VALUES, a, None, None, n, C.byref(out), w, need - 1) == S.ERR_WORKSPACE
    assert call(S.SUM_VALUES, a, None, None, n, C.byref(out), C.c_void_p((1 << 20) + 64), need) == S.ERR_WORKSPACE
