"""Pins of the oracle's mosaic (Sect. 4, second experiment; Table 2 / Table 6): geometry against
the paper's example, split/stitch as exact inverses, the one-tile mosaic as the plain
reconstruction, and the delta-PSF mosaic reaching the known minimiser."""
import numpy as np
import pytest

from oracle import sgp_oracle as O


def test_paper_example_geometry():
    # a 256 x 256 image, four partially overlapping 160 x 160 sub-domains, 128 x 128 pieces kept
    assert O.mosaic_axis(256, 2, 160) == [(0, 160, 0, 128), (96, 256, 128, 256)]


@pytest.mark.parametrize("N,n,s", [(256, 2, 160), (256, 3, 100), (96, 4, 40), (100, 1, 100), (64, 2, 33)])
def test_pieces_partition_the_axis_inside_their_windows(N, n, s):
    ax = O.mosaic_axis(N, n, s)
    assert ax[0][0] == 0 and ax[-1][1] == N                     # first/last sub-domain at the edges
    assert ax[0][2] == 0 and ax[-1][3] == N
    for k, (w0, w1, c0, c1) in enumerate(ax):
        assert w1 - w0 == s and w0 <= c0 < c1 <= w1
        if k:
            assert c0 == ax[k - 1][3]                            # contiguous, non-overlapping


def test_impossible_geometry_is_rejected():
    with pytest.raises(ValueError):
        O.mosaic_axis(256, 2, 100)                               # piece [0, 128) exceeds [0, 100)
    with pytest.raises(ValueError):
        O.mosaic_axis(64, 2, 80)


def test_split_then_stitch_is_identity():
    rng = np.random.default_rng(0)
    g = rng.random((2, 72, 60))
    n, sub, ext = (3, 2), (32, 36), (48, 48)
    tiles, masks = O.mosaic_split(g, n, sub, ext)
    assert tiles.shape == (6, 2, 48, 48) and masks.shape == (6, 48, 48)
    assert np.all(masks.sum(axis=(1, 2)) == 32 * 36)
    assert np.all(tiles[:, :, masks[0] == 0] == 0)             # zero padding outside M_S
    for j in range(2):
        np.testing.assert_array_equal(O.mosaic_stitch(tiles[:, j], (72, 60), n, sub, ext), g[j])


def _gauss(N, sigma):
    y, x = np.mgrid[:N, :N]
    k = np.exp(-((y - N // 2) ** 2 + (x - N // 2) ** 2) / (2 * sigma ** 2))
    return k / k.sum()


def test_one_tile_mosaic_is_the_plain_reconstruction():
    """sub = ext = the image: M_S = 1 everywhere, so boundary SGP is periodic SGP (Sect. 2.4 with
    all masks one) and the mosaic is that reconstruction."""
    rng = np.random.default_rng(1)
    N = 32
    f = rng.random((N, N)) * 200
    psf = _gauss(N, 1.5)
    g = rng.poisson(O.conv_periodic(f, O.prepare_psf(psf)) + 5.0).astype(np.float64)
    mos = O.mosaic(psf[None], g[None], [5.0], n=(1, 1), sub=(N, N), ext=(N, N), n_iter=15)
    ref = O.sgp(O.Problem(psf[None], g[None], [5.0]), stop=O.StopRule("fixed", max_iter=15)).f
    np.testing.assert_allclose(mos, ref, rtol=1e-9, atol=1e-9 * ref.max())


def test_delta_psf_mosaic_reaches_the_minimiser():
    """With K = delta the KL objective separates per pixel; on S its minimiser is g - b (g > b
    here), and every piece lies inside its sub-domain's S, so the mosaic converges to g - b."""
    rng = np.random.default_rng(2)
    H, W = 40, 36
    g = rng.poisson(100.0, (H, W)).astype(np.float64) + 30.0
    b = 5.0
    E = 32
    delta = np.zeros((E, E))
    delta[E // 2, E // 2] = 1.0
    mos = O.mosaic(delta[None], g[None], [b], n=(2, 2), sub=(24, 24), ext=(E, E), method="sgp", n_iter=60)
    np.testing.assert_allclose(mos, g - b, rtol=1e-6)
    mos_rl = O.mosaic(delta[None], g[None], [b], n=(2, 2), sub=(24, 24), ext=(E, E), method="rl", n_iter=400)
    np.testing.assert_allclose(mos_rl, g - b, rtol=1e-4)
