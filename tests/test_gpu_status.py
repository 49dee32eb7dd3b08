"""Failure statuses of the solver, provoked from the host side with finite, valid inputs.

  * SGP_ERR_LINESEARCH: a first step length of 1e5 with at most one Armijo reduction (Algorithm 1,
    step 5; the 30-reduction cap is a reading, the cap itself a parameter): neither lambda = 1 nor
    lambda = theta decreases J, so the solve stops at f^(0) with the line-search status, as the
    oracle does.
  * SGP_ERR_TIMEOUT: a discrepancy level (Sect. 3.3, Eq. discrepancy) that two iterations cannot
    reach: the solve returns the status after exactly two iterations, with the iterate of two
    fixed iterations.
  * SGP_ERR_NONFINITE: a user start of 1e36 per pixel (finite in FP32) whose transform overflows,
    so the KL value at the start is not finite: the set-up controller stops the problem with the
    status and the start is kept.
Every case returns through the C ABI with the context still usable: a later valid solve runs.
"""
import numpy as np
import pytest

from oracle import sgp_oracle as O
from paper_1210_2258_b300 import scenes
from tests.gpu_util import dev, gpu_problem, host, oracle_problem, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stars64():
    return scenes.stars_scene(seed=4, N=64, n_stars=10)


def test_linesearch_failure_status(gpu, stars64):
    sc = stars64
    orc = oracle_problem(sc)
    ref = O.sgp(orc, P=O.SGPParams(alpha0=1e5, max_backtracks=1), stop=O.StopRule("fixed", max_iter=5))
    assert ref.status == "linesearch" and ref.iters == 0
    prob = gpu_problem(gpu, sc, gpu.default_params(alpha0=1e5, max_backtracks=1))
    f0 = host(prob.get_f())
    iters = prob.solve_until(gpu.STOP_DISCREPANCY, max_iter=5, eta=0.5, raise_on_error=False)
    assert prob.last_status == gpu.ERR_LINESEARCH, prob.last_status
    info = prob.info()
    assert info.status == gpu.ERR_LINESEARCH and info.k == 0 and iters == [0]
    f = host(prob.get_f())
    assert np.array_equal(f, f0)                       # the iterate is kept
    assert rel_l2(f, ref.f) <= 1e-6


def test_timeout_status(gpu, stars64):
    sc = stars64
    orc = oracle_problem(sc)
    ref = O.sgp(orc, stop=O.StopRule("fixed", max_iter=2))
    prob = gpu_problem(gpu, sc)
    iters = prob.solve_until(gpu.STOP_DISCREPANCY, max_iter=2, eta=0.5, raise_on_error=False)
    assert prob.last_status == gpu.ERR_TIMEOUT, prob.last_status
    info = prob.info()
    assert info.k == 2 and iters == [2] and info.status == 0
    assert rel_l2(host(prob.get_f()), ref.f) <= 1e-5
    assert abs(prob.kl_value() - ref.J) <= 1e-5 * ref.J
    # the context stays usable: continue to a level the scene reaches
    more = prob.solve_until(gpu.STOP_DISCREPANCY, max_iter=500, eta=1.5)
    assert 0 < more[0] < 500


def test_nonfinite_status_from_an_overflowing_start(gpu, stars64):
    sc = stars64
    prob = gpu_problem(gpu, sc)
    big = np.full(sc.shape, 1e36, np.float32)
    prob.set_start(0, gpu.START_USER, dev(big))
    iters = prob.solve_until(gpu.STOP_DISCREPANCY, max_iter=10, eta=1.0, raise_on_error=False)
    assert prob.last_status == gpu.ERR_NONFINITE, prob.last_status
    info = prob.info()
    assert info.status == gpu.ERR_NONFINITE and info.k == 0 and iters == [0]
    assert np.array_equal(host(prob.get_f()), big.astype(np.float64))
    # a fresh context on the same device still solves
    ok = gpu_problem(gpu, sc)
    assert ok.solve_until(gpu.STOP_DISCREPANCY, max_iter=500, eta=1.5)[0] > 0


def test_user_start_from_a_temporary_view_is_read_in_stream_order(gpu, stars64):
    """sgp_set_start is asynchronous (stream-ordered): a start given as a non-contiguous view is
    copied by the binding, and the solve sees that start even when the view is dropped and its
    memory is reused right after the call."""
    import torch
    sc = stars64
    start = np.random.default_rng(5).uniform(1.0, 2.0, sc.shape).astype(np.float32)
    ref = gpu_problem(gpu, sc)
    ref.set_start(0, gpu.START_USER, dev(start))
    it_ref = ref.solve_until(gpu.STOP_DISCREPANCY, max_iter=30, eta=1.5, raise_on_error=False)
    f_ref = host(ref.get_f())

    prob = gpu_problem(gpu, sc)
    view = dev(np.ascontiguousarray(start.T)).t()          # the same values, not contiguous
    assert not view.is_contiguous()
    prob.set_start(0, gpu.START_USER, view)
    del view
    junk = [torch.full(sc.shape, 7.0, device="cuda") for _ in range(8)]   # reuse of freed memory
    it = prob.solve_until(gpu.STOP_DISCREPANCY, max_iter=30, eta=1.5, raise_on_error=False)
    del junk
    assert it == it_ref and it[0] > 0 and prob.last_status == ref.last_status
    assert np.array_equal(host(prob.get_f()), f_ref)


def test_setup_failure_of_one_problem_in_a_batch(gpu, stars64):
    """The solve loop starts without reading the set-up status back: a problem whose set-up fails
    (the overflowing start above) stops with its status at iteration 0 while the other problem of
    the same context solves exactly as it does alone."""
    sc = stars64
    psf = dev(np.asarray(sc.psfs, np.float32))
    b = list(np.asarray(sc.b, np.float32))
    g = dev(np.asarray(sc.g, np.float32))
    alone = gpu_problem(gpu, sc)
    it_alone = alone.solve_until(gpu.STOP_DISCREPANCY, max_iter=500, eta=1.5)
    pair = gpu.Problems([psf, psf], [b, b])
    pair.set_data(0, g)
    pair.set_data(1, g)
    pair.set_start(0, gpu.START_USER, dev(np.full(sc.shape, 1e36, np.float32)))
    it = pair.solve_until(gpu.STOP_DISCREPANCY, max_iter=500, eta=1.5, raise_on_error=False)
    assert pair.last_status == gpu.ERR_NONFINITE
    assert pair.info(0).status == gpu.ERR_NONFINITE and it[0] == 0
    assert pair.info(1).status == 0 and it[1] == it_alone[0]
    assert np.array_equal(host(pair.get_f(1)), host(alone.get_f()))
