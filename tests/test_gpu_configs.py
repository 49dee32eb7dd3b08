"""Parity at the full sizes of the multi-view and batched workloads.

  * three views of 1024 x 1024 (a 300-source star cluster with a diffuse nebula, two-pupil
    interferometric PSFs at 0, 60 and 120 degrees, b = 20): multiple RL and SGP (Sect. 2.3,
    Algorithm 1) against the FP64 oracle, and the convergence stop of Eq. (convergence), the rule
    the paper uses for this kind of multi-view star-cluster problem (Sect. 4, Table 7);
  * a mixed-size batch of boundary problems whose largest, 1024 x 1024 cut from a 1.5x larger
    scene, is reconstructed on its 1536 x 1536 extended domain (Sect. 2.4) in the same launches as
    a 384 and a 128 problem.
The oracle's transforms run on every host core here (same arithmetic as numpy.fft, split over rows)."""
import os

import numpy as np
import pytest

from oracle import sgp_oracle as O
from paper_1210_2258_b300 import scenes
from tests.gpu_util import dev, gpu_problem, host, oracle_problem, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def threaded_oracle():
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    O.set_fft_workers(n)
    yield
    O.set_fft_workers(None)


@pytest.fixture(scope="module")
def cluster1024():
    return scenes.cluster_multiview_scene(seed=0, N=1024)


def test_multiview_1024_rl_and_sgp_match_oracle(gpu, cluster1024):
    sc = cluster1024
    orc = oracle_problem(sc)
    n_rl, n_sgp = 10, 8
    ref_rl = O.rl(orc, stop=O.StopRule("fixed", max_iter=n_rl))
    rl = gpu_problem(gpu, sc)
    rl.rl_iterate(n_rl)
    assert rel_l2(host(rl.get_f()), ref_rl.f) <= 1e-3
    assert abs(rl.kl_value() - ref_rl.J) <= 1e-5 * ref_rl.J
    ref = O.sgp(orc, stop=O.StopRule("fixed", max_iter=n_sgp))
    sg = gpu_problem(gpu, sc)
    sg.sgp_iterate(n_sgp)
    assert rel_l2(host(sg.get_f()), ref.f) <= 1e-3
    assert abs(sg.kl_value() - ref.J) <= 1e-5 * ref.J
    tr = sg.trace()
    assert [int(x) for x in tr[:n_sgp, 5]] == [t["backtracks"] for t in ref.trace]
    assert [int(x) for x in tr[:n_sgp, 6]] == [t["branch"] for t in ref.trace]


def test_multiview_1024_convergence_stop_fires(gpu, cluster1024):
    """The discrepancy of this scene never falls to 1 (the band-limited PSFs leave the noise
    outside their support unfitted); Eq. (convergence) with tol = 1e-3 stops where the oracle
    does (the first 30 iterations are inside the reproducible horizon)."""
    sc = cluster1024
    tol = 1e-3
    ref = O.sgp(oracle_problem(sc), stop=O.StopRule("convergence", max_iter=400, tol=tol))
    assert ref.iters < 400
    sg = gpu_problem(gpu, sc)
    it = sg.solve_until(gpu.STOP_CONVERGENCE, max_iter=400, tol=tol)[0]
    assert sg.info().stopped == 1 and it < 400
    if ref.iters <= 30:
        assert it == ref.iters, (it, ref.iters)
    else:
        assert abs(it - ref.iters) <= max(3, ref.iters // 10), (it, ref.iters)
    tr = sg.trace()
    J = tr[:it, 1]
    assert abs(J[-1] - J[-2]) <= tol * J[-2] and np.all(np.abs(np.diff(J[:-1])) > tol * J[:-2])


def test_batch_with_1536_padded_problem(gpu):
    rng = scenes.rng_for(21)
    scs = [scenes.boundary_scene(rng, 1024, 2.0, 20.0), scenes.boundary_scene(rng, 384, 3.0, 10.0),
           scenes.boundary_scene(rng, 128, 1.5, 40.0)]
    assert scs[0].g.shape[-1] == 1536 and len({s.g.shape for s in scs}) == 3
    prob = gpu.Problems([dev(np.asarray(s.psfs, np.float32)) for s in scs],
                        [list(np.asarray(s.b, np.float32)) for s in scs], [dev(s.mask) for s in scs])
    for i, s in enumerate(scs):
        prob.set_data(i, dev(np.asarray(s.g, np.float32)))
    n = 8
    prob.sgp_iterate(n)
    for i, s in enumerate(scs):
        ref = O.sgp(oracle_problem(s), stop=O.StopRule("fixed", max_iter=n))
        assert prob.info(i).k == n
        assert rel_l2(host(prob.get_f(i)), ref.f) <= 1e-3, i
        assert abs(prob.kl_value(i) - ref.J) <= 1e-5 * ref.J, (i, prob.kl_value(i), ref.J)
