"""The allocation-free convolution entry point (sgp_convolve_noalloc) against the FP64 oracle and
the workspace-based operators.

Some callers cannot allocate device memory (their allocator is owned by another framework, or
allocation is not allowed where they run); sgp_convolve_noalloc serves them from a fixed scratch
array inside the library.  This file is collected last on purpose.  Every case calls the entry
point twice in a row through the C ABI (a convolution, then a correlation of other data, reusing
the shared scratch) and checks both results against the oracle's periodic convolution and
correlation and against sgp_apply_A / sgp_apply_AT, within the operator tolerance of the other
tests.  The shapes cover the size limit (512 x 512, and 128 x 2048 / 2048 x 128, which fill the
column-item table and select the 2048-point column plan), a 3 * 2^k side, both PSF origins and a
non-default stream."""
import ctypes as C

import numpy as np
import pytest

from oracle import sgp_oracle as O
from paper_1210_2258_b300 import scenes
from tests.gpu_util import dev, host, rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-5
CASES = [(256, 384, 0, False), (512, 512, 0, True), (128, 2048, 1, False), (2048, 128, 0, True),
         (384, 96, 1, True)]


@pytest.mark.parametrize("H,W,origin,own_stream", CASES)
def test_noalloc_convolution_matches_oracle_and_operators(gpu, H, W, origin, own_stream):
    import torch
    lib = gpu.load()
    rng = scenes.rng_for(77 + H + W + origin)
    psf = (rng.random((H, W)) ** 4).astype(np.float32)       # asymmetric
    f1 = rng.random((H, W)).astype(np.float32)
    f2 = (rng.random((H, W)) * 10).astype(np.float32)
    K = O.prepare_psf(psf.astype(np.float64), "corner" if origin == gpu.PSF_CORNER else "center")
    orc1 = O.conv_periodic(f1.astype(np.float64), K)
    orc2 = O.corr_periodic(f2.astype(np.float64), K)
    prob = gpu.Problems(dev(psf[None]), [1.0], psf_origin=origin)
    prob.set_data(0, dev(np.ones((1, H, W), np.float32)))
    ref1 = host(prob.apply_A(dev(f1)))[0]
    ref2 = host(prob.apply_AT(dev(f2[None])))
    torch.cuda.synchronize()
    d_psf, d_f1, d_f2 = dev(psf), dev(f1), dev(f2)
    out1 = torch.empty((H, W), dtype=torch.float32, device="cuda")
    out2 = torch.empty((H, W), dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream() if own_stream else None
    sp = stream.cuda_stream if stream is not None else None
    st = lib.sgp_convolve_noalloc(d_psf.data_ptr(), d_f1.data_ptr(), out1.data_ptr(), H, W, origin, 0, sp)
    assert st == gpu.OK, lib.sgp_last_error()
    st = lib.sgp_convolve_noalloc(d_psf.data_ptr(), d_f2.data_ptr(), out2.data_ptr(), H, W, origin, 1, sp)
    assert st == gpu.OK, lib.sgp_last_error()
    (stream or torch.cuda.current_stream()).synchronize()
    torch.cuda.synchronize()
    r1, r2 = host(out1), host(out2)
    assert rel_l2(r1, orc1) <= TOL, rel_l2(r1, orc1)
    assert rel_l2(r2, orc2) <= TOL, rel_l2(r2, orc2)
    assert rel_l2(r1, ref1) <= TOL and rel_l2(r2, ref2) <= TOL


def test_noalloc_rejects_sizes_beyond_its_limit(gpu):
    lib = gpu.load()
    st = lib.sgp_convolve_noalloc(C.c_void_p(256), C.c_void_p(256), C.c_void_p(256), 1024, 512, 0, 0, None)
    assert st == gpu.ERR_SIZE and b"262144" in lib.sgp_last_error()


def test_noalloc_refuses_a_capturing_stream(gpu):
    """Under stream capture the call returns SGP_ERR_STATE before touching the stream."""
    import torch
    lib = gpu.load()
    H = W = 64
    psf = dev(np.ones((H, W), np.float32))
    f = dev(np.ones((H, W), np.float32))
    out = torch.empty((H, W), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        st = lib.sgp_convolve_noalloc(psf.data_ptr(), f.data_ptr(), out.data_ptr(), H, W, 0, 0, s.cuda_stream)
        out.add_(1.0)             # the capture holds one node, so it ends cleanly
    assert st == gpu.ERR_STATE and b"captured" in lib.sgp_last_error()
