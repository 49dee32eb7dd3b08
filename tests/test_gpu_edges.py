"""Edge cases: non-square tiny multi-view problems, the largest view count, degenerate data (an
all-zero image, whose one-RL-step set-up has no positive pixel, Sect. 3.2), and a batch in which
one problem fails its set-up while the others iterate."""
import numpy as np
import pytest

from oracle import sgp_oracle as O
from paper_1210_2258_b300 import scenes
from tests.gpu_util import dev, gpu_problem, host, oracle_problem, rel_l2

pytestmark = pytest.mark.gpu


def test_non_square_tiny_multi_view(gpu):
    rng = scenes.rng_for(11)
    H, W, p = 24, 48, 2
    f = scenes.star_field(rng, H, W, 12) + 5.0
    psfs = np.stack([scenes.gaussian_psf(H, W, s) for s in (1.0, 1.7)])
    g = np.stack([scenes.poisson(rng, scenes.blur_periodic(f, psfs[j]) + 3.0) for j in range(p)])
    sc = scenes.Scene(psfs=psfs, g=g, b=np.array([3.0, 3.0]), f_true=f)
    orc = oracle_problem(sc)
    ref_rl = O.rl(orc, stop=O.StopRule("fixed", max_iter=30))
    rl = gpu_problem(gpu, sc)
    rl.rl_iterate(30)
    assert rel_l2(host(rl.get_f()), ref_rl.f) <= 1e-3
    assert abs(rl.kl_value() - ref_rl.J) <= 1e-5 * ref_rl.J
    ref = O.sgp(orc, stop=O.StopRule("fixed", max_iter=10))
    sg = gpu_problem(gpu, sc)
    sg.sgp_iterate(10)
    assert rel_l2(host(sg.get_f()), ref.f) <= 1e-3
    assert abs(sg.kl_value() - ref.J) <= 1e-5 * ref.J


def test_largest_view_count_operators(gpu):
    rng = scenes.rng_for(12)
    H = W = 32
    p = 8
    psfs = np.stack([scenes.gaussian_psf(H, W, 0.8 + 0.3 * j) for j in range(p)]).astype(np.float32)
    g = rng.random((p, H, W)).astype(np.float32) + 1.0
    prob = gpu.Problems(dev(psfs), [1.0] * p)
    prob.set_data(0, dev(g))
    orc = O.Problem(psfs.astype(np.float64), g.astype(np.float64), np.ones(p))
    f = rng.random((H, W)).astype(np.float32)
    y = rng.random((p, H, W)).astype(np.float32)
    Af = host(prob.apply_A(dev(f)))
    for j in range(p):
        assert rel_l2(Af[j], orc.A(j, f.astype(np.float64))) <= 1e-5
    ATy = host(prob.apply_AT(dev(y)))
    assert rel_l2(ATy, sum(orc.AT(j, y[j].astype(np.float64)) for j in range(p))) <= 1e-5
    with pytest.raises(gpu.SGPError):
        gpu.Problems(dev(np.concatenate([psfs, psfs[:1]])), [1.0] * 9)   # 9 views: above the limit


def test_all_zero_image_is_a_set_up_error(gpu):
    H = W = 32
    psf = scenes.gaussian_psf(H, W, 1.5).astype(np.float32)[None]
    g = np.zeros((1, H, W), np.float32)
    with pytest.raises(ValueError):
        O.sgp(O.Problem(psf.astype(np.float64), g.astype(np.float64), np.array([2.0])),
              stop=O.StopRule("fixed", max_iter=3))
    prob = gpu.Problems(dev(psf), [2.0])
    prob.set_data(0, dev(g))
    with pytest.raises(gpu.SGPError) as e:
        prob.sgp_iterate(3)
    assert e.value.status == gpu.ERR_ARG


def test_failed_problem_does_not_stop_the_batch(gpu):
    H = W = 64
    good = scenes.stars_scene(seed=3, N=H, n_stars=10)
    psf = np.asarray(good.psfs, np.float32)
    batch = gpu.Problems([dev(psf), dev(psf)], [[float(good.b[0])], [float(good.b[0])]])
    batch.set_data(0, dev(np.zeros((1, H, W), np.float32)))
    batch.set_data(1, dev(np.asarray(good.g, np.float32)))
    batch.sgp_iterate(15)
    assert batch.info(0).status == gpu.ERR_ARG and batch.info(0).k == 0
    assert batch.info(1).status == 0 and batch.info(1).k == 15
    single = gpu_problem(gpu, good)
    single.sgp_iterate(15)
    assert rel_l2(host(batch.get_f(1)), host(single.get_f())) <= 1e-5
