"""Precision of the library's FP64-grade sums ("mixed" variant) at 2048 x 2048.

The KL value J_0 (Eq. KL), the four scaled-BB sums (Eq. BB1, BB2) and the Armijo differences
(Algorithm 1, step 5) are sums of FP32 pixel terms.  sgp_sum_terms computes those terms with the
device functions of the iteration passes and sums them with the passes' reduction; here the terms
come from a real state of the 2048^2 galaxy workload (two consecutive SGP iterates, their
gradients, the projected direction and A d) and the library's sums are compared with the exact
(correctly rounded, math.fsum) sum of the very same FP32 terms.  The mixed variant must agree to
1e-12 of the exact sum; the plain-FP32 variant is reported for contrast and is far coarser.
"""
import math

import numpy as np
import pytest

from paper_1210_2258_b300 import scenes
from tests.gpu_util import dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def state2048(gpu):
    import torch
    sc = scenes.galaxy_scene(seed=0, N=2048)
    b = float(sc.b[0])
    prob = gpu.Problems(dev(sc.psfs.astype(np.float32)), [b])
    g = dev(sc.g.astype(np.float32))
    prob.set_data(0, g)
    prob.sgp_iterate(4)
    f4 = prob.get_f().clone()
    prob.sgp_iterate(1)
    f5 = prob.get_f().clone()
    info = prob.info()
    g0 = g[0]

    def grad(f):
        u = prob.apply_A(f)[0] + b
        r = torch.where(u > 0, g0 / u, torch.zeros_like(u))
        return 1.0 - prob.apply_AT(r[None].contiguous()), u

    gr5, u5 = grad(f5)
    gr4, _ = grad(f4)
    D = torch.clamp(f5, float(info.L1), float(info.L2))
    d = torch.clamp(f5 - float(info.alpha) * D * gr5, min=0.0) - f5
    Ad = prob.apply_A(d.contiguous())[0]
    torch.cuda.synchronize()
    return {"g": g0.contiguous(), "u": u5.contiguous(), "s": (f5 - f4).contiguous(), "z": (gr5 - gr4).contiguous(),
            "D": D.contiguous(), "Ad": Ad.contiguous()}


CASES = [("KL", 1, ("g", "u", None), 1.0), ("ARMIJO", 2, ("g", "u", "Ad"), 1.0), ("ARMIJO", 2, ("g", "u", "Ad"), 0.4),
         ("BB s2/D2", 3, ("s", "z", "D"), 1.0), ("BB sz/D", 4, ("s", "z", "D"), 1.0),
         ("BB szD", 5, ("s", "z", "D"), 1.0), ("BB z2D2", 6, ("s", "z", "D"), 1.0)]


@pytest.mark.parametrize("name,kind,args,lam", CASES)
def test_mixed_sums_match_exact_sum_of_the_same_fp32_terms(gpu, state2048, name, kind, args, lam):
    st = state2048
    a, b, c = (st[k] if k else None for k in args)
    mixed, terms = gpu.sum_terms(kind, a, b, c, lam=lam, reduce_fp64=1)
    plain, terms_p = gpu.sum_terms(kind, a, b, c, lam=lam, reduce_fp64=0)
    t = terms.double().cpu().numpy().ravel()
    assert np.array_equal(t, terms_p.double().cpu().numpy().ravel())   # same terms in both variants
    assert np.all(np.isfinite(t)) and t.size == 2048 * 2048
    exact = math.fsum(t.tolist())
    absum = float(np.sum(np.abs(t)))
    err_mixed, err_plain = abs(mixed - exact), abs(plain - exact)
    print(f"{name} lam={lam}: exact {exact:.17g}, sum|t|/|sum| {absum / abs(exact):.3g}, "
          f"mixed rel {err_mixed / abs(exact):.3g}, plain rel {err_plain / abs(exact):.3g}")
    assert err_mixed <= 1e-12 * abs(exact), (name, err_mixed / abs(exact))
    assert err_mixed <= 1e-13 * absum
