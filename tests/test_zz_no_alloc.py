"""The allocation-free convolution entry point (sgp_convolve_noalloc) against the workspace-based
operators.

Some callers cannot allocate device memory (their allocator is owned by another framework, or
allocation is not allowed where they run); sgp_convolve_noalloc serves them from a fixed scratch
array inside the library.  This file is collected last on purpose: it checks, through the C ABI,
two consecutive calls (convolution, then correlation with different inputs, reusing the shared
scratch) against sgp_apply_A / sgp_apply_AT within the operator tolerance of the other tests."""
import ctypes as C

import numpy as np
import pytest

from paper_1210_2258_b300 import scenes
from tests.gpu_util import dev, host, rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-5


def test_noalloc_convolution_matches_workspace_operators(gpu):
    import torch
    lib = gpu.load()
    H, W = 256, 384
    rng = scenes.rng_for(77)
    psf = (rng.random((H, W)) ** 4).astype(np.float32)       # asymmetric
    f1 = rng.random((H, W)).astype(np.float32)
    f2 = (rng.random((H, W)) * 10).astype(np.float32)
    prob = gpu.Problems(dev(psf[None]), [1.0])
    prob.set_data(0, dev(np.ones((1, H, W), np.float32)))
    ref1 = host(prob.apply_A(dev(f1)))[0]
    ref2 = host(prob.apply_AT(dev(f2[None])))
    d_psf, d_f1, d_f2 = dev(psf), dev(f1), dev(f2)
    out = torch.empty((H, W), dtype=torch.float32, device="cuda")
    st = lib.sgp_convolve_noalloc(d_psf.data_ptr(), d_f1.data_ptr(), out.data_ptr(), H, W, gpu.PSF_CENTER, 0, None)
    assert st == gpu.OK, lib.sgp_last_error()
    torch.cuda.synchronize()
    assert rel_l2(host(out), ref1) <= TOL
    st = lib.sgp_convolve_noalloc(d_psf.data_ptr(), d_f2.data_ptr(), out.data_ptr(), H, W, gpu.PSF_CENTER, 1, None)
    assert st == gpu.OK, lib.sgp_last_error()
    torch.cuda.synchronize()
    assert rel_l2(host(out), ref2) <= TOL


def test_noalloc_rejects_sizes_beyond_its_limit(gpu):
    lib = gpu.load()
    st = lib.sgp_convolve_noalloc(C.c_void_p(256), C.c_void_p(256), C.c_void_p(256), 1024, 512, 0, 0, None)
    assert st == gpu.ERR_SIZE and b"262144" in lib.sgp_last_error()
