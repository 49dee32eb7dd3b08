"""GPU parity of the imaging operators A_j f and sum_j A_j^T y_j (Sect. 2.2-2.4, Eq. projection and
backprojection) against the FP64 oracle: relative l2 error <= 1e-5 at every supported transform
shape class, with asymmetric random PSFs, several views, both PSF origins and boundary masks."""
import numpy as np
import pytest

from oracle import sgp_oracle as O
from paper_1210_2258_b300 import scenes
from tests.gpu_util import dev, host, rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-5

CASES = [
    # H, W, p, origin, boundary
    (16, 16, 1, "center", False),
    (16, 24, 2, "corner", False),
    (24, 32, 1, "center", False),      # 232 idle rows in the single row item (ragged)
    (48, 64, 3, "center", False),
    (96, 128, 1, "corner", False),
    (256, 48, 1, "center", False),     # 24 packed columns in a 32-column tile (ragged)
    (128, 192, 2, "center", False),
    (384, 256, 1, "center", False),
    (512, 768, 1, "corner", False),
    (1024, 96, 3, "center", False),
    (1536, 64, 1, "center", False),
    (2048, 32, 1, "center", False),
    (32, 2048, 1, "center", False),
    (64, 64, 1, "center", True),
    (192, 192, 2, "center", True),
    # planes of 1024 or more rows store the spectrum interleaved by groups of 4 rows
    (1024, 192, 2, "corner", True),
    (1536, 384, 2, "center", True),
    (2048, 96, 1, "center", True),
]


def _random_problem(H, W, p, boundary, seed):
    rng = scenes.rng_for(seed)
    psfs = rng.random((p, H, W)) ** 4          # asymmetric, positive
    psfs /= psfs.sum(axis=(1, 2), keepdims=True)
    if boundary:
        psfs = np.stack([scenes.gaussian_psf(H, W, 1.5 + j) for j in range(p)])
        psfs = psfs * (1.0 + 0.3 * rng.random((p, H, W)))    # break the symmetry
    g = rng.poisson(20.0, (p, H, W)).astype(np.float64)
    mask = None
    if boundary:
        mask = np.zeros((H, W), np.uint8)
        mask[H // 4:H - H // 4, W // 5:W - W // 6] = 1
    return psfs.astype(np.float32), g.astype(np.float32), mask


@pytest.mark.parametrize("H,W,p,origin,boundary", CASES)
def test_operators_match_oracle(gpu, H, W, p, origin, boundary):
    psfs, g, mask = _random_problem(H, W, p, boundary, seed=H * 7 + W + p)
    rng = scenes.rng_for(H + W)
    f = rng.random((H, W)).astype(np.float32)
    y = rng.random((p, H, W)).astype(np.float32)
    org = gpu.PSF_CENTER if origin == "center" else gpu.PSF_CORNER
    prob = gpu.Problems(dev(psfs), [3.0] * p, dev(mask) if mask is not None else None, psf_origin=org)
    prob.set_data(0, dev(g))
    Af = host(prob.apply_A(dev(f)))
    ATy = host(prob.apply_AT(dev(y)))
    orc = O.Problem(psfs.astype(np.float64), g.astype(np.float64), [3.0] * p, mask_S=mask, origin=origin)
    for j in range(p):
        ref = orc.A(j, f.astype(np.float64))
        assert rel_l2(Af[j], ref) <= TOL, (j, rel_l2(Af[j], ref))
    ref = sum(orc.AT(j, y[j].astype(np.float64)) for j in range(p))
    assert rel_l2(ATy, ref) <= TOL, rel_l2(ATy, ref)


def test_adjoint_identity_on_gpu(gpu):
    psfs, g, mask = _random_problem(128, 96, 2, True, seed=3)
    prob = gpu.Problems(dev(psfs), [1.0, 1.0], dev(mask))
    prob.set_data(0, dev(g))
    rng = scenes.rng_for(9)
    f = rng.random((128, 96)).astype(np.float32)
    y = rng.random((2, 128, 96)).astype(np.float32)
    lhs = float(np.sum(host(prob.apply_A(dev(f))) * y))
    rhs = float(np.sum(f * host(prob.apply_AT(dev(y)))))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_full_size_airy_operator(gpu):
    """2048 x 2048 with the Airy PSF of the single-image benchmark workload."""
    N = 2048
    psf = scenes.airy_psf(N).astype(np.float32)
    rng = scenes.rng_for(11)
    f = (rng.random((N, N)) * 100).astype(np.float32)
    prob = gpu.Problems(dev(psf[None]), [50.0])
    prob.set_data(0, dev(np.full((1, N, N), 60.0, np.float32)))
    Af = host(prob.apply_A(dev(f)))[0]
    K = O.prepare_psf(psf.astype(np.float64))
    assert rel_l2(Af, O.conv_periodic(f.astype(np.float64), K)) <= TOL
    ATy = host(prob.apply_AT(dev(f[None])))
    assert rel_l2(ATy, O.corr_periodic(f.astype(np.float64), K)) <= TOL


def test_delta_psf_is_identity(gpu):
    H, W = 64, 48
    psf = np.zeros((1, H, W), np.float32)
    psf[0, H // 2, W // 2] = 1.0
    prob = gpu.Problems(dev(psf), [0.0])
    prob.set_data(0, dev(np.ones((1, H, W), np.float32)))
    f = scenes.rng_for(2).random((H, W)).astype(np.float32)
    assert np.max(np.abs(host(prob.apply_A(dev(f)))[0] - f)) < 1e-5


def test_invalid_psf_and_data_are_rejected(gpu):
    import torch
    H = W = 32
    bad = -np.ones((1, H, W), np.float32)
    with pytest.raises(gpu.SGPError) as e:
        gpu.Problems(dev(bad), [1.0])
    assert e.value.status == gpu.ERR_PSF
    psf = scenes.gaussian_psf(H, W, 1.0).astype(np.float32)[None]
    prob = gpu.Problems(dev(psf), [1.0])
    g = np.ones((1, H, W), np.float32)
    g[0, 3, 4] = np.nan
    with pytest.raises(gpu.SGPError) as e:
        prob.set_data(0, dev(g))
    assert e.value.status == gpu.ERR_NONFINITE
    with pytest.raises(gpu.SGPError):
        prob.sgp_iterate(1)          # no valid data yet
