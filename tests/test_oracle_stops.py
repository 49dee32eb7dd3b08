"""Pins of the oracle's starting point (Sect. 3.1) and stopping rules (Sect. 3.3) (CPU only).

The references here do not come from the oracle:
  * the constant start c = mean_j (sum_S g_j - sum_S b_j) / |S| on R is summed pixel by pixel in
    plain Python over hand-built problems whose R is known in advance (a delta PSF gives
    alpha_j = M_S, so R = S);
  * with a delta PSF the operator A is the identity, so RL is the scalar recursion
    f_{k+1} = f_k g / (f_k + b) at every pixel and J_k, D_k and the reconstruction error are
    closed-form sums of its values: the iteration at which the convergence, discrepancy and
    minimum-error rules fire, and the iterate each returns, are known before the oracle runs;
  * for SGP, whose iterates have no closed form, the stop index of a rule is read off a FIXED run
    of the same problem (which never evaluates a stop rule), and the minimum-error rule is checked
    against errors computed from fixed runs of every length.
Each pin is a helper that raises AssertionError; the last tests plant mistakes in the oracle
(a start that forgets b or divides by H W, a convergence test against the wrong J) and check that
the pins catch them.
"""
import math

import numpy as np
import pytest

from oracle import sgp_oracle as O
from paper_1210_2258_b300 import scenes


def _delta_psf(H, W):
    k = np.zeros((H, W))
    k[H // 2, W // 2] = 1.0
    return k


# ----------------------------------------------------------------- constant start (Sect. 3.1)
def _boundary_two_view_problem():
    H, W = 16, 16
    rng = scenes.rng_for(40)
    mask = np.zeros((H, W), np.uint8)
    mask[3:13, 2:14] = 1                       # |S| = 120, not H W
    g = np.stack([rng.integers(0, 20, (H, W)), rng.integers(5, 40, (H, W))]).astype(np.float64)
    g[:, mask == 0] = 1000.0                   # junk outside S must not count
    b = np.stack([np.full((H, W), 1.5), rng.random((H, W)) * 4.0])
    psfs = np.stack([_delta_psf(H, W)] * 2)
    return psfs, g, b, mask


def _expected_constant(g, b, mask):
    """mean over views of (sum over S of g - sum over S of b) / |S|, summed pixel by pixel."""
    p, H, W = g.shape
    nS = sum(1 for r in range(H) for c in range(W) if mask[r, c])
    per_view = []
    for j in range(p):
        sg = sum(float(g[j, r, c]) for r in range(H) for c in range(W) if mask[r, c])
        sb = sum(float(b[j, r, c]) for r in range(H) for c in range(W) if mask[r, c])
        per_view.append((sg - sb) / nS)
    return sum(per_view) / p


def check_constant_start(make_start):
    """make_start(psfs, g, b, mask) -> f0 of the oracle (mask None: periodic)."""
    # boundary, two views: the value on R = S, zero outside
    psfs, g, b, mask = _boundary_two_view_problem()
    c = _expected_constant(g, b, mask)
    f0 = make_start(psfs, g, b, mask)
    assert np.allclose(f0[mask == 1], c, rtol=1e-14, atol=0.0), (f0[mask == 1][:3], c)
    assert np.all(f0[mask == 0] == 0.0)
    # periodic: S is the whole array
    full = np.ones(mask.shape, np.uint8)
    c_full = _expected_constant(g, b, full)
    f0 = make_start(psfs, g, b, None)
    assert np.allclose(f0, c_full, rtol=1e-14, atol=0.0), (f0[0, 0], c_full)
    # c <= 0: the fallback max(mean of g over S, 1e-3)
    gb = np.full((1, 8, 8), 3.0)
    f0 = make_start(_delta_psf(8, 8)[None], gb, np.full((1, 8, 8), 3.0), None)
    assert np.all(f0 == 3.0)
    f0 = make_start(_delta_psf(8, 8)[None], np.zeros((1, 8, 8)), np.full((1, 8, 8), 3.0), None)
    assert np.all(f0 == 1e-3)


def _oracle_constant(psfs, g, b, mask):
    return O.Problem(psfs, g, b, mask_S=mask).initial("constant")


def test_constant_start_pinned():
    check_constant_start(_oracle_constant)


# ----------------------------------------------------------------- RL with a delta PSF (closed form)
def _delta_problem(seed=41, H=16, W=16, b=2.0):
    rng = scenes.rng_for(seed)
    truth = rng.random((H, W)) * 30.0
    g = rng.poisson(truth + b).astype(np.float64)
    return O.Problem(_delta_psf(H, W)[None], g[None], [b]), g, b


def _scalar_rl(g, b, f0, n):
    """f_{k+1} = f_k g / (f_k + b) pixel by pixel (RL with A = identity), k = 0..n."""
    fs = [np.array(f0, np.float64)]
    for _ in range(n):
        f = fs[-1]
        fs.append(np.array([[f[r, c] * g[r, c] / (f[r, c] + b) for c in range(f.shape[1])]
                            for r in range(f.shape[0])]))
    return fs


def _scalar_kl(g, b, f):
    tot = 0.0
    for r in range(g.shape[0]):
        for c in range(g.shape[1]):
            u = f[r, c] + b
            gv = g[r, c]
            tot += (gv * math.log(gv / u) if gv > 0 else 0.0) + u - gv
    return tot


def test_rl_delta_psf_follows_the_scalar_recursion():
    prob, g, b = _delta_problem()
    f0 = prob.initial("constant")
    fs = _scalar_rl(g, b, f0, 6)
    res = O.rl(prob, stop=O.StopRule("fixed", max_iter=6))
    np.testing.assert_allclose(res.f, fs[6], rtol=1e-12, atol=1e-12)
    for k, t in enumerate(res.trace, start=1):
        assert abs(t["J"] - _scalar_kl(g, b, fs[k])) <= 1e-12 * t["J"]


def check_rl_convergence_stop(rl_fn):
    prob, g, b = _delta_problem()
    f0 = prob.initial("constant")
    fs = _scalar_rl(g, b, f0, 60)
    Js = [_scalar_kl(g, b, f) for f in fs]
    tol = 2e-3
    # Eq. (convergence): first k >= 1 with |J_k - J_{k-1}| <= tol J_{k-1}
    k_exp = next(k for k in range(1, 61) if abs(Js[k] - Js[k - 1]) <= tol * Js[k - 1])
    assert 3 <= k_exp <= 55
    ratio = abs(Js[k_exp] - Js[k_exp - 1]) / Js[k_exp - 1]
    assert ratio < tol * (1 - 1e-6)           # not a rounding-level decision
    res = rl_fn(prob, O.StopRule("convergence", max_iter=60, tol=tol))
    assert res.iters == k_exp, (res.iters, k_exp)
    np.testing.assert_allclose(res.f, fs[k_exp], rtol=1e-12, atol=1e-12)


def check_rl_discrepancy_stop(rl_fn):
    prob, g, b = _delta_problem()
    f0 = prob.initial("constant")
    fs = _scalar_rl(g, b, f0, 200)
    nS = g.size
    Ds = [2.0 * _scalar_kl(g, b, f) / nS for f in fs]
    eta = 0.5 * (Ds[0] + Ds[-1])               # a level the run crosses
    k_exp = next(k for k in range(1, 201) if Ds[k] <= eta)
    res = rl_fn(prob, O.StopRule("discrepancy", max_iter=200, eta=eta))
    assert res.iters == k_exp, (res.iters, k_exp)
    np.testing.assert_allclose(res.f, fs[k_exp], rtol=1e-12, atol=1e-12)


def check_rl_min_error_stop(rl_fn):
    prob, g, b = _delta_problem()
    f0 = prob.initial("constant")
    fs = _scalar_rl(g, b, f0, 12)
    f_true = fs[5]                             # the error is smallest (zero) at k = 5
    err = [np.linalg.norm(f - f_true) for f in fs]
    assert all(err[k] < err[k - 1] for k in range(1, 6)) and err[6] > err[5]
    res = rl_fn(prob, O.StopRule("min_error", max_iter=12, f_true=f_true))
    assert res.iters == 5, res.iters               # the error grew at k = 6: return f^(5)
    np.testing.assert_allclose(res.f, fs[5], rtol=1e-12, atol=1e-12)


def _oracle_rl(prob, stop):
    return O.rl(prob, stop=stop)


def test_rl_convergence_stop_pinned():
    check_rl_convergence_stop(_oracle_rl)


def test_rl_discrepancy_stop_pinned():
    check_rl_discrepancy_stop(_oracle_rl)


def test_rl_min_error_stop_returns_previous_iterate():
    check_rl_min_error_stop(_oracle_rl)


# ----------------------------------------------------------------- SGP stop branches
def _sgp_problem():
    sc = scenes.stars_scene(seed=3, N=32, n_stars=6)
    return O.Problem(sc.psfs, sc.g, sc.b)


def test_sgp_convergence_stop_matches_fixed_run():
    prob = _sgp_problem()
    n = 60
    fixed = O.sgp(prob, stop=O.StopRule("fixed", max_iter=n))
    Js = [prob.kl(prob.initial("constant"))] + [t["J"] for t in fixed.trace]
    tol = 1e-3
    k_exp = next(k for k in range(1, n + 1) if abs(Js[k] - Js[k - 1]) <= tol * Js[k - 1])
    assert 2 <= k_exp < n
    res = O.sgp(prob, stop=O.StopRule("convergence", max_iter=n, tol=tol))
    assert res.iters == k_exp
    ref = O.sgp(prob, stop=O.StopRule("fixed", max_iter=k_exp))
    assert np.array_equal(res.f, ref.f)


def test_sgp_min_error_stop_returns_previous_iterate():
    prob = _sgp_problem()
    f_true = O.sgp(prob, stop=O.StopRule("fixed", max_iter=6)).f
    fs = [prob.initial("constant")] + [O.sgp(prob, stop=O.StopRule("fixed", max_iter=k)).f for k in range(1, 12)]
    rho = [np.linalg.norm(f - f_true) / np.linalg.norm(f_true) for f in fs]
    k_up = next(k for k in range(1, 12) if rho[k] > rho[k - 1])   # first increase of the error
    res = O.sgp(prob, stop=O.StopRule("min_error", max_iter=11, f_true=f_true))
    assert res.iters == k_up - 1
    assert np.array_equal(res.f, fs[k_up - 1])


# ----------------------------------------------------------------- planted mistakes are caught
def test_planted_constant_start_mistakes_are_caught():
    def forgets_b(psfs, g, b, mask):
        prob = O.Problem(psfs, g, b, mask_S=mask)
        c = float(np.mean([prob.g[j][prob.MS > 0].sum() / prob.nS for j in range(prob.p)]))
        return c * prob.MR

    def divides_by_array_size(psfs, g, b, mask):
        prob = O.Problem(psfs, g, b, mask_S=mask)
        c = float(np.mean([(prob.g[j].sum() - prob.b[j].sum()) / (prob.H * prob.W) for j in range(prob.p)]))
        return c * prob.MR

    def everywhere(psfs, g, b, mask):
        return np.full(g.shape[1:], float(np.max(_oracle_constant(psfs, g, b, mask))))

    for wrong in (forgets_b, divides_by_array_size, everywhere):
        with pytest.raises(AssertionError):
            check_constant_start(wrong)


def test_planted_stop_mistakes_are_caught(monkeypatch):
    real = O._stop_check

    def against_new_J(rule, k, J_old, J_new, D_new):      # |J_k - J_{k-1}| <= tol J_k, one step late
        if rule.kind == "convergence":
            return k >= 2 and abs(J_new - J_old) <= rule.tol * J_new * 0.5
        return real(rule, k, J_old, J_new, D_new)

    monkeypatch.setattr(O, "_stop_check", against_new_J)
    with pytest.raises(AssertionError):
        check_rl_convergence_stop(_oracle_rl)

    def returns_current(prob, stop):                      # min-error rule keeping the worse iterate
        if stop.kind != "min_error":
            return O.rl(prob, stop=stop)
        res = O.rl(prob, stop=stop)
        return O.rl(prob, stop=O.StopRule("fixed", max_iter=res.iters + 1))

    monkeypatch.setattr(O, "_stop_check", real)
    with pytest.raises(AssertionError):
        check_rl_min_error_stop(returns_current)
