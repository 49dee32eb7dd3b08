"""Pins of the regularised SGP of the oracle (CPU): J_0 + beta/2 ||f||^2 with the split-gradient
(SGM) scaling (Sect. 5; the regulariser itself is a reading, the paper names none).

  * beta = 0 is exactly the unregularised method;
  * the gradient against central finite differences of J_0 + R;
  * the split grad = V - U with V, U >= 0, and the defining property of the SGM scaling: a unit step
    along -D grad without clipping is the multiplicative step f U / V;
  * with a delta PSF every pixel is a one-dimensional problem whose minimiser is the non-negative
    root of beta f^2 + (1 + beta b) f + b - g = 0, which SGP must reach;
  * the Armijo decrease of J_0 + R along the run, and the KKT conditions at convergence.
"""
import numpy as np
import pytest

from oracle import sgp_oracle as O
from paper_1210_2258_b300 import scenes


def _small(seed=31, N=24, b=3.0):
    rng = scenes.rng_for(seed)
    f = scenes.star_field(rng, N, N, 6) + 2.0
    psf = scenes.gaussian_psf(N, N, 1.5)
    g = scenes.poisson(rng, scenes.blur_periodic(f, psf) + b)
    return O.Problem(psf[None], g[None], [b])


def test_beta_zero_is_the_plain_method():
    prob = _small()
    a = O.sgp(prob, stop=O.StopRule("fixed", max_iter=15))
    b = O.sgp(prob, P=O.SGPParams(reg_beta=0.0), stop=O.StopRule("fixed", max_iter=15))
    assert np.array_equal(a.f, b.f) and [t["J"] for t in a.trace] == [t["J"] for t in b.trace]


def test_regularised_gradient_matches_finite_differences():
    prob = _small(N=12)
    beta = 0.05
    rng = np.random.default_rng(3)
    f = prob.initial() * (1.0 + 0.5 * rng.random((prob.H, prob.W)))
    obj = lambda x: prob.kl(x) + O.reg_value(x, beta)
    V, U = O.sgm_split(prob, f, beta)
    grad = V - U
    np.testing.assert_allclose(grad, prob.grad(f) + beta * f, rtol=1e-12, atol=1e-12)
    for (i, j) in [(0, 0), (3, 7), (11, 5), (6, 6)]:
        h = 1e-4 * f[i, j]
        e = np.zeros_like(f)
        e[i, j] = h
        fd = (obj(f + e) - obj(f - e)) / (2 * h)
        assert abs(fd - grad[i, j]) <= 1e-6 * max(1.0, abs(grad[i, j])), (i, j, fd, grad[i, j])


def test_sgm_scaling_unit_step_is_the_multiplicative_step():
    prob = _small()
    beta = 0.2
    f = prob.initial() * (0.5 + np.random.default_rng(4).random((prob.H, prob.W)))
    V, U = O.sgm_split(prob, f, beta)
    assert np.all(V > 0) and np.all(U >= 0)
    D = O.sgm_scaling(prob, f, 0.0, np.inf, beta)      # no clipping
    y = f - D * (V - U)
    np.testing.assert_allclose(y, f * U / V, rtol=1e-12, atol=1e-12)
    assert np.all(y >= 0)
    np.testing.assert_allclose(O.sgm_scaling(prob, f, 0.0, np.inf, 0.0), prob.w * f, rtol=0, atol=0)


@pytest.mark.parametrize("beta", [0.01, 0.3])
def test_delta_psf_minimiser_is_the_root_of_the_pixel_quadratic(beta):
    N, b = 16, 4.0
    rng = scenes.rng_for(33)
    g = rng.poisson(rng.random((N, N)) * 40.0 + b).astype(np.float64)
    psf = np.zeros((N, N))
    psf[N // 2, N // 2] = 1.0
    prob = O.Problem(psf[None], g[None], [b])
    q1 = 1.0 + beta * b
    f_star = np.maximum(0.0, (-q1 + np.sqrt(q1 * q1 - 4.0 * beta * (b - g))) / (2.0 * beta))
    res = O.sgp(prob, P=O.SGPParams(reg_beta=beta), stop=O.StopRule("convergence", max_iter=3000, tol=1e-14))
    np.testing.assert_allclose(res.f, f_star, rtol=1e-5, atol=1e-6)
    # the regulariser pulls every pixel below the unregularised minimiser max(g - b, 0)
    assert np.all(f_star <= np.maximum(g - b, 0.0) + 1e-12)


def test_regularised_run_descends_and_meets_kkt():
    prob = _small()
    beta = 0.02
    res = O.sgp(prob, P=O.SGPParams(reg_beta=beta), stop=O.StopRule("convergence", max_iter=4000, tol=1e-13))
    objs = [t["J"] + t["R"] for t in res.trace]
    assert all(b <= a + 1e-12 * abs(a) for a, b in zip(objs, objs[1:]))
    f = res.f
    grad = prob.grad(f) + beta * f
    pos = f > 1e-6 * f.max()
    assert np.max(np.abs(grad[pos])) <= 1e-4 * np.max(np.abs(grad))  # stationarity on the support
    assert np.all(grad[~pos] >= -1e-6 * np.max(np.abs(grad)))        # no descent into the bound
    assert np.all(f >= 0)


def test_planted_sign_error_in_the_regulariser_is_caught(monkeypatch):
    real = O.sgm_split

    def wrong(prob, f, beta):
        V, U = real(prob, f, beta)
        return V - 2 * beta * f, U          # grad = ... - beta f: the sign of the term flipped

    monkeypatch.setattr(O, "sgm_split", wrong)
    with pytest.raises(AssertionError):
        test_regularised_gradient_matches_finite_differences()
