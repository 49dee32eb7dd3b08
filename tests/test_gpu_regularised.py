"""GPU regularised SGP (J_0 + beta/2 ||f||^2 with the split-gradient scaling; reading of Sect. 5)
against the FP64 oracle, and against the closed-form minimiser of the delta-PSF problem."""
import numpy as np
import pytest

from oracle import sgp_oracle as O
from paper_1210_2258_b300 import scenes
from tests.gpu_util import dev, gpu_problem, host, oracle_problem, rel_l2

pytestmark = pytest.mark.gpu


def _f32(x):
    return float(np.float32(x))


@pytest.mark.parametrize("beta", [1e-7, 1e-5])
def test_regularised_sgp_matches_oracle_stars_256(gpu, beta):
    sc = scenes.stars_scene(seed=0, N=256)
    n = 20
    orc = oracle_problem(sc)
    ref = O.sgp(orc, P=O.SGPParams(reg_beta=_f32(beta)), stop=O.StopRule("fixed", max_iter=n))
    prob = gpu_problem(gpu, sc, gpu.default_params(reg_beta=beta))
    prob.sgp_iterate(n)
    info = prob.info()
    assert info.k == n
    assert rel_l2(host(prob.get_f()), ref.f) <= 1e-3
    assert abs(info.J - ref.J) <= 1e-5 * ref.J, (info.J, ref.J)
    R = ref.trace[-1]["R"]
    assert R > 1e-3 * ref.J                           # the term matters at this beta
    assert abs(info.reg - R) <= 1e-5 * R, (info.reg, R)
    tr = prob.trace()
    assert [int(x) for x in tr[:n, 5]] == [t["backtracks"] for t in ref.trace]
    assert [int(x) for x in tr[:n, 6]] == [t["branch"] for t in ref.trace]
    # the regularised iterate differs from the unregularised one
    plain = O.sgp(orc, stop=O.StopRule("fixed", max_iter=n))
    assert rel_l2(ref.f, plain.f) > 1e-3


def test_regularised_boundary_sgp_matches_oracle(gpu):
    sc = scenes.boundary_scene(scenes.rng_for(9), 96, 2.0, 10.0)
    beta = 1e-5
    n = 15
    ref = O.sgp(oracle_problem(sc), P=O.SGPParams(reg_beta=_f32(beta)), stop=O.StopRule("fixed", max_iter=n))
    prob = gpu_problem(gpu, sc, gpu.default_params(reg_beta=beta))
    prob.sgp_iterate(n)
    assert rel_l2(host(prob.get_f()), ref.f) <= 1e-3
    assert abs(prob.kl_value() - ref.J) <= 1e-5 * ref.J


def test_regularised_delta_psf_reaches_the_pixel_quadratic_root(gpu):
    """With a delta PSF each pixel minimises g ln(g/(f+b)) + f + b - g + beta f^2/2: f* is the
    non-negative root of beta f^2 + (1 + beta b) f + b - g = 0 (no oracle involved)."""
    N, b, beta = 64, 4.0, 0.05
    rng = scenes.rng_for(34)
    g = rng.poisson(rng.random((N, N)) * 60.0 + b).astype(np.float32)
    psf = np.zeros((N, N), np.float32)
    psf[N // 2, N // 2] = 1.0
    prob = gpu.Problems(dev(psf[None]), [b], params=gpu.default_params(reg_beta=beta))
    prob.set_data(0, dev(g[None]))
    prob.solve_until(gpu.STOP_CONVERGENCE, max_iter=3000, tol=1e-9)
    bb = np.float64(_f32(beta))
    q1 = 1.0 + bb * b
    f_star = np.maximum(0.0, (-q1 + np.sqrt(q1 * q1 - 4.0 * bb * (b - g.astype(np.float64)))) / (2.0 * bb))
    f = host(prob.get_f())
    assert np.max(np.abs(f - f_star)) <= 1e-3 * np.max(f_star), np.max(np.abs(f - f_star))


def test_regularised_convergence_stop_matches_oracle(gpu):
    sc = scenes.stars_scene(seed=5, N=64, n_stars=12)
    beta, tol = 1e-6, 1e-3
    ref = O.sgp(oracle_problem(sc), P=O.SGPParams(reg_beta=_f32(beta)),
                stop=O.StopRule("convergence", max_iter=500, tol=tol))
    prob = gpu_problem(gpu, sc, gpu.default_params(reg_beta=beta))
    it = prob.solve_until(gpu.STOP_CONVERGENCE, max_iter=500, tol=tol)[0]
    assert ref.iters < 60 and it == ref.iters, (it, ref.iters)


def test_rl_refuses_regularisation(gpu):
    sc = scenes.stars_scene(seed=1, N=32, n_stars=4)
    prob = gpu_problem(gpu, sc, gpu.default_params(reg_beta=1e-3))
    with pytest.raises(gpu.SGPError) as e:
        prob.rl_iterate(2)
    assert e.value.status == gpu.ERR_ARG
