"""Problems of different sizes advancing together in the same launches (multi-size passes):
boundary-corrected problems cut from larger scenes, each compared with the FP64 oracle."""
import numpy as np
import pytest

from oracle import sgp_oracle as O
from paper_1210_2258_b300 import scenes
from tests.gpu_util import dev, host, oracle_problem, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    return scenes.boundary_batch(seed=3, count=5, sides=(48, 64, 96, 128))


def _make(gpu, scs, params=None):
    prob = gpu.Problems([dev(np.asarray(s.psfs, np.float32)) for s in scs],
                        [list(np.asarray(s.b, np.float32)) for s in scs],
                        [dev(s.mask) for s in scs], params)
    for i, s in enumerate(scs):
        prob.set_data(i, dev(np.asarray(s.g, np.float32)))
    return prob


def test_batch_has_mixed_sizes(batch):
    assert len({s.g.shape for s in batch}) >= 2


def test_mixed_batch_rl_and_sgp_match_oracle(gpu, batch):
    prob = _make(gpu, batch)
    prob.rl_iterate(20)
    prob2 = _make(gpu, batch)
    prob2.sgp_iterate(12)
    for i, s in enumerate(batch):
        orc = oracle_problem(s)
        ref = O.rl(orc, stop=O.StopRule("fixed", max_iter=20))
        assert rel_l2(host(prob.get_f(i)), ref.f) <= 1e-3, i
        assert abs(prob.kl_value(i) - ref.J) <= 1e-5 * ref.J, i
        ref2 = O.sgp(orc, stop=O.StopRule("fixed", max_iter=12))
        assert rel_l2(host(prob2.get_f(i)), ref2.f) <= 1e-3, i
        assert abs(prob2.kl_value(i) - ref2.J) <= 1e-5 * ref2.J, i


def test_mixed_batch_discrepancy_stop_per_problem(gpu, batch):
    prob = _make(gpu, batch)
    its = prob.solve_until(gpu.STOP_DISCREPANCY, max_iter=2000, eta=1.0, raise_on_error=False)
    for i, s in enumerate(batch):
        ref = O.sgp(oracle_problem(s), stop=O.StopRule("discrepancy", max_iter=2000, eta=1.0))
        info = prob.info(i)
        if ref.iters <= 60:         # inside the horizon where SGP trajectories are reproducible
            assert abs(its[i] - ref.iters) <= 2, (i, its[i], ref.iters)
        if ref.iters < 2000:        # the oracle reaches the stop: so must every GPU problem
            assert its[i] < 2000 and info.D <= 1.0, (i, its[i], info.D)
