"""GPU parity of OSEM (Sect. 2.3, Algorithm 2 with Eq. OSEMstep; Sect. 2.4, Eq. boundaryOSEM)
against the FP64 oracle on the same seeded inputs.

OSEM is a fixed-count multiplicative iteration like RL (no step-length or line-search decisions),
so FP32 and FP64 trajectories stay close: after 10 iterations (10 p view updates) the
reconstruction is held to 1e-4 relative l2 and the KL value to 1e-5 relative."""
import numpy as np
import pytest

from oracle import sgp_oracle as O
from paper_1210_2258_b300 import scenes
from tests.gpu_util import dev, gpu_problem, host, oracle_problem, rel_l2

pytestmark = pytest.mark.gpu


def _masked(base, margin):
    """The same views detected on a centred sub-square only: M_S = 1 there, g = 0 outside."""
    H, W = base.g.shape[-2:]
    mask = np.zeros((H, W), np.uint8)
    mask[margin:H - margin, margin:W - margin] = 1
    return scenes.Scene(psfs=base.psfs, g=base.g * mask, b=base.b, f_true=base.f_true, mask=mask,
                        meta=dict(kind="boundary-multiview"))


@pytest.mark.parametrize("p", [2, 3])
def test_osem_periodic_matches_oracle(gpu, p):
    sc = scenes.cluster_multiview_scene(seed=4, N=128, p=p, n_sources=40)
    orc = oracle_problem(sc)
    ref = O.osem(orc, n_iter=10)
    prob = gpu_problem(gpu, sc)
    prob.osem_iterate(10)
    f = host(prob.get_f())
    assert rel_l2(f, ref.f) <= 1e-4, rel_l2(f, ref.f)
    assert abs(prob.kl_value() - ref.J) <= 1e-5 * ref.J, (prob.kl_value(), ref.J)
    assert prob.info().k == 10 * p
    assert np.all(f >= 0)


def test_boundary_osem_matches_oracle(gpu):
    sc = _masked(scenes.cluster_multiview_scene(seed=6, N=96, p=2, n_sources=30), 12)
    orc = oracle_problem(sc)
    ref = O.osem(orc, n_iter=8)
    prob = gpu_problem(gpu, sc)
    prob.osem_iterate(8)
    f = host(prob.get_f())
    assert rel_l2(f, ref.f) <= 1e-4, rel_l2(f, ref.f)
    assert abs(prob.kl_value() - ref.J) <= 1e-5 * ref.J
    assert np.all(f[orc.MR == 0] == 0) and np.all(f >= 0)


def test_osem_batch_of_equal_sizes(gpu):
    """Two problems in one context: each launch covers view j of both (view-major item lists)."""
    scs = [scenes.cluster_multiview_scene(seed=s, N=96, p=3, n_sources=25) for s in (7, 8)]
    prob = gpu.Problems([dev(np.asarray(s.psfs, np.float32)) for s in scs],
                        [list(np.asarray(s.b, np.float32)) for s in scs])
    for i, s in enumerate(scs):
        prob.set_data(i, dev(np.asarray(s.g, np.float32)))
    prob.osem_iterate(6)
    for i, s in enumerate(scs):
        orc = oracle_problem(s)
        ref = O.osem(orc, n_iter=6)
        assert rel_l2(host(prob.get_f(i)), ref.f) <= 1e-4
        assert abs(prob.kl_value(i) - ref.J) <= 1e-5 * ref.J


def test_osem_one_view_is_rl_and_resumes(gpu):
    """p = 1: OSEM is RL (Algorithm 2 with one subset); two calls continue where the first ended."""
    sc = scenes.stars_scene(seed=1, N=128, n_stars=30)
    a = gpu_problem(gpu, sc)
    a.osem_iterate(6)
    b = gpu_problem(gpu, sc)
    b.rl_iterate(6)
    fa = host(a.get_f())
    assert rel_l2(fa, host(b.get_f())) <= 1e-6
    c = gpu_problem(gpu, sc)
    c.osem_iterate(2)
    c.osem_iterate(4)
    assert rel_l2(host(c.get_f()), fa) <= 1e-6
    # RL continues from the OSEM result
    c.rl_iterate(3)
    ref = O.rl(oracle_problem(sc), f0=O.osem(oracle_problem(sc), n_iter=6).f, stop=O.StopRule("fixed", max_iter=3))
    assert rel_l2(host(c.get_f()), ref.f) <= 1e-4


def test_osem_rejects_mixed_sizes(gpu):
    rng = scenes.rng_for(3)
    scs = [scenes.boundary_scene(rng, 48, 1.5, 10.0), scenes.boundary_scene(rng, 64, 1.5, 10.0)]
    assert scs[0].g.shape != scs[1].g.shape
    prob = gpu.Problems([dev(np.asarray(s.psfs, np.float32)) for s in scs],
                        [list(np.asarray(s.b, np.float32)) for s in scs], [dev(s.mask) for s in scs])
    for i, s in enumerate(scs):
        prob.set_data(i, dev(np.asarray(s.g, np.float32)))
    with pytest.raises(gpu.SGPError):
        prob.osem_iterate(1)


def test_osem_with_psf_band(gpu):
    """3 x 512^2 two-pupil views: the PSF band drops about half of the spectrum columns, and the
    OSEM sub-steps run over it."""
    sc = scenes.cluster_multiview_scene(seed=9, N=512, p=3, n_sources=80)
    orc = oracle_problem(sc)
    ref = O.osem(orc, n_iter=4)
    prob = gpu_problem(gpu, sc)
    assert prob.info().band_cols < 256
    prob.osem_iterate(4)
    assert rel_l2(host(prob.get_f()), ref.f) <= 1e-4
    assert abs(prob.kl_value() - ref.J) <= 1e-5 * ref.J
