"""Deep Armijo backtracking (Algorithm 1, step 5): a large first step length alpha_0 makes the
first iteration reject lambda = 1, theta, .., theta^3, so the extra pass (theta^4 .. theta^30) has
to decide; the decisions and the KL value must follow the FP64 oracle, through the fixed-count
graphs and through the device-side solve loop."""
import numpy as np
import pytest

from oracle import sgp_oracle as O
from paper_1210_2258_b300 import scenes
from tests.gpu_util import gpu_problem, host, oracle_problem, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("alpha0", [300.0, 1e4])
def test_deep_backtracking_follows_the_oracle(gpu, alpha0):
    sc = scenes.stars_scene(seed=2, N=64, n_stars=12)
    orc = oracle_problem(sc)
    ref = O.sgp(orc, P=O.SGPParams(alpha0=alpha0), stop=O.StopRule("fixed", max_iter=8))
    bt_ref = [t["backtracks"] for t in ref.trace]
    assert bt_ref[0] > 3
    params = gpu.default_params(alpha0=alpha0)
    for solve in ("iterate", "loop"):
        prob = gpu_problem(gpu, sc, params)
        if solve == "iterate":
            prob.sgp_iterate(8)
        else:
            prob.solve_until(gpu.STOP_FIXED, max_iter=8)
        tr = prob.trace()
        assert list(tr[:8, 5].astype(int)) == bt_ref, (solve, tr[:8, 5], bt_ref)
        assert abs(tr[0, 4] - ref.trace[0]["lam"]) <= 1e-12
        assert abs(prob.kl_value() - ref.J) <= 1e-5 * ref.J
        assert rel_l2(host(prob.get_f()), ref.f) <= 1e-3
