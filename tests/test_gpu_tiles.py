"""The autotuned row tile: every candidate tile gives the oracle's iteration (parity within the SGP
horizon with the KL bound of the FP32-transform envelope, RL over 200 iterations at 1e-5), the autotuner picks a candidate, and contexts of one size share
its choice (so a batch and a single problem still agree bit for bit)."""
import numpy as np
import pytest

from oracle import sgp_oracle as O
from paper_1210_2258_b300 import scenes
from tests.gpu_util import fp32_envelope, gpu_problem, host, oracle_problem, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stars256():
    return scenes.stars_scene(seed=0, N=256)


def test_every_row_tile_matches_the_oracle(gpu, stars256):
    sc = stars256
    orc = oracle_problem(sc)
    n = 30
    ref = O.sgp(orc, stop=O.StopRule("fixed", max_iter=n))
    ref_rl = O.rl(orc, stop=O.StopRule("fixed", max_iter=200))
    T = 256 // 32                       # 256 columns: 128 complex per row, 16 per thread -> 8 threads
    seen = []
    for R in (32, 16, 8, 4):            # 256-thread tile down to 32-thread blocks
        prob = gpu_problem(gpu, sc)
        prob.set_tile(R)
        assert prob.tile() == (R, R * T)
        prob.sgp_iterate(n)
        assert prob.info().k == n
        assert abs(prob.kl_value() - ref.J) <= fp32_envelope()[1][n - 1] * ref.J, (R, prob.kl_value(), ref.J)
        f = host(prob.get_f())
        assert rel_l2(f, ref.f) <= 1e-3
        seen.append(f)
        rl = gpu_problem(gpu, sc)
        rl.set_tile(R)
        rl.rl_iterate(200)
        assert rel_l2(host(rl.get_f()), ref_rl.f) <= 1e-3
        assert abs(rl.kl_value() - ref_rl.J) <= 1e-5 * ref_rl.J
    # the tiles differ only in the grouping of the partial sums
    for f in seen[1:]:
        assert rel_l2(f, seen[0]) <= 1e-4
    with pytest.raises(gpu.SGPError):
        gpu_problem(gpu, sc).set_tile(3)
    with pytest.raises(gpu.SGPError):
        gpu_problem(gpu, sc).set_tile(2)     # 16-thread blocks: below one warp


def test_autotuner_choice_is_a_candidate_and_shared(gpu):
    sc = scenes.stars_scene(seed=7, N=192, n_stars=20)
    a = gpu_problem(gpu, sc)
    a.sgp_iterate(2)
    R, threads = a.tile()
    # 192 columns: 96 complex per row, 24 per thread -> 4 threads per row, 64 rows per 256 threads
    assert R in (64, 32, 16, 8) and threads == 4 * R
    b = gpu_problem(gpu, sc)
    b.sgp_iterate(2)
    assert b.tile() == (R, threads)
    assert np.array_equal(host(a.get_f()), host(b.get_f()))
