"""Mosaic of boundary-corrected reconstructions (Sect. 4, second experiment; Table 2 / Table 6):
the library's geometry (host code) against the oracle's, and on the GPU the split / stitch kernels
(bit-exact copies) and whole mosaics of SGP, RL and OSEM against the FP64 oracle's mosaic."""
import numpy as np
import pytest

from oracle import sgp_oracle as O
from paper_1210_2258_b300 import scenes
from tests.gpu_util import dev, host, rel_l2

CASES = [((256, 256), (2, 2), (160, 160), (256, 256)), ((128, 96), (2, 3), (80, 48), (128, 64)),
         ((100, 100), (1, 1), (100, 100), (128, 128)), ((90, 200), (3, 4), (40, 60), (48, 64))]


@pytest.mark.parametrize("shape,n,sub,ext", CASES)
def test_library_geometry_matches_oracle(shape, n, sub, ext):
    """Host code only (no GPU): the library's sub-domains and pieces equal the oracle's."""
    from paper_1210_2258_b300 import mosaic
    gy, gx = mosaic.geometry(shape[0], shape[1], n, sub, ext)
    assert gy == O.mosaic_axis(shape[0], n[0], sub[0])
    assert gx == O.mosaic_axis(shape[1], n[1], sub[1])


def test_library_rejects_impossible_geometry():
    from paper_1210_2258_b300 import mosaic, sgp
    with pytest.raises(sgp.SGPError):
        mosaic.geometry(256, 256, (2, 2), (100, 100), (256, 256))   # pieces of 128 > sub-domains
    with pytest.raises(sgp.SGPError):
        mosaic.geometry(64, 64, (2, 2), (40, 40), (32, 32))          # sub-domain larger than the array


def _scene(N=128, sigma=1.5, b=8.0, seed=11):
    rng = scenes.rng_for(seed)
    f = scenes.star_field(rng, N, N, 40) + scenes.sersic_galaxy(rng, N, N, n_profiles=2, peak=2e3)
    psf = scenes.gaussian_psf(N, N, sigma)
    g = scenes.poisson(rng, scenes.blur_periodic(f, psf) + b)
    return f, psf, g, b


@pytest.mark.gpu
def test_split_and_stitch_kernels_are_exact(gpu):
    import torch
    from paper_1210_2258_b300 import mosaic
    rng = np.random.default_rng(3)
    for shape, n, sub, ext in CASES:
        g = rng.random((2,) + shape).astype(np.float32)
        m = gpu.Mosaic(shape[0], shape[1], n[0], n[1], sub[0], sub[1], ext[0], ext[1])
        nt = n[0] * n[1]
        tiles = torch.full((nt, 2) + ext, 7.0, device="cuda")
        masks = torch.full((nt,) + ext, 9, dtype=torch.uint8, device="cuda")
        gd = dev(g)
        import ctypes as C
        gpu._check(gpu.load().sgp_mosaic_split(C.byref(m), 2, gd.data_ptr(), tiles.data_ptr(), masks.data_ptr(), None))
        t_ref, m_ref = O.mosaic_split(g.astype(np.float64), n, sub, ext)
        np.testing.assert_array_equal(host(tiles), t_ref)
        np.testing.assert_array_equal(masks.cpu().numpy(), m_ref)
        out = torch.full(shape, -1.0, device="cuda")
        recs = tiles[:, 1].contiguous()
        gpu._check(gpu.load().sgp_mosaic_stitch(C.byref(m), recs.data_ptr(), out.data_ptr(), None))
        np.testing.assert_array_equal(host(out), g[1].astype(np.float64))


@pytest.mark.gpu
@pytest.mark.parametrize("method,n_iter", [("sgp", 25), ("rl", 30), ("osem", 20)])
def test_mosaic_matches_oracle(gpu, method, n_iter):
    from paper_1210_2258_b300 import mosaic
    f, psf, g, b = _scene()
    n, sub, ext = (2, 2), (80, 80), (128, 128)
    g32 = np.asarray(g, np.float32)
    psf32 = np.asarray(psf, np.float32)
    ref = O.mosaic(psf32.astype(np.float64)[None], g32.astype(np.float64)[None], [b], n, sub, ext, method, n_iter)
    ms = mosaic.MosaicSolver(dev(psf32)[None], dev(g32)[None], [b], n, sub, ext)
    out = host(ms.solve(method, n_iter))
    assert rel_l2(out, ref) <= 1e-3, rel_l2(out, ref)
    assert np.all(out >= 0)
