"""CPU checks of the rewritten pixel formulas the CUDA passes use, against the literal definitions.

They pin the mathematics (FP64 numpy), not the kernels: the GPU parity tests compare the kernels
with the oracle.  Formulas:
  KL term (Eq. KL):  g ln(g/u) + u - g = (u - g) z - 2 g z^3 S(z^2),  z = (u - g)/(u + g),
                     S(w) = sum_k w^k/(2k+3), truncated after w^6 where 1/2 < u/g < 2.
  Armijo pixel difference (Alg. 1 step 5):
                     g ln(u/(u + lam A d)) + lam A d = (u - g) q + g phi(q),  q = lam A d / u,
                     phi(q) = q - ln(1 + q), series for |q| < 1/8 truncated after q^9.
"""
import numpy as np


def kl_literal(g, u):
    return g * np.log(g / u) + u - g


def kl_zseries(g, u, terms=7):
    z = (u - g) / (u + g)
    w = z * z
    S = np.zeros_like(z)
    for k in reversed(range(terms)):
        S = S * w + 1.0 / (2 * k + 3)
    return (u - g) * z - 2.0 * g * z ** 3 * S


def test_kl_zseries_matches_definition():
    rng = np.random.default_rng(0)
    g = rng.uniform(1.0, 1e4, 20000)
    u = g * rng.uniform(0.5, 2.0, g.size)           # the series' range
    ref = kl_literal(g, u)
    got = kl_zseries(g, u)
    rel = np.abs(got - ref) / np.maximum(ref, 1e-300)
    assert np.max(rel[ref > 1e-6 * g]) < 5e-8
    # where the literal form cancels (u -> g) the series keeps full relative accuracy
    u2 = g * (1.0 + rng.uniform(-1e-4, 1e-4, g.size))
    exact = g * ((u2 - g) / g) ** 2 / 2                # leading term of the expansion
    assert np.allclose(kl_zseries(g, u2), exact, rtol=2e-4)


def test_kl_zseries_truncation_is_what_matters():
    # at the edge of the range (u/g -> 2) the 7-term series is within 5e-9; two terms fewer is not
    # within 5e-8, so a dropped coefficient is caught
    g = np.array([100.0])
    u = np.array([199.0])
    rel = lambda n: abs(kl_zseries(g, u, n)[0] - kl_literal(g, u)[0]) / kl_literal(g, u)[0]
    assert rel(7) < 5e-9
    assert rel(5) > 5e-8


def phi_series(q, nmax=9):
    out = np.zeros_like(q)
    for n in range(2, nmax + 1):
        out += (-q) ** n / n
    return out


def test_armijo_pixel_difference():
    rng = np.random.default_rng(1)
    n = 20000
    g = rng.poisson(200.0, n).astype(float) + 1.0
    u = g * rng.uniform(0.8, 1.25, n)
    ad = u * rng.uniform(-0.3, 0.3, n)
    for lam in [1.0, 0.4, 0.16, 0.064]:
        q = lam * ad / u
        ref = g * np.log(u / (u + lam * ad)) + lam * ad
        phi = np.where(np.abs(q) < 0.125, phi_series(q), q - np.log1p(q))
        got = (u - g) * q + g * phi
        assert np.allclose(got, ref, rtol=1e-7, atol=1e-9 * np.abs(lam * ad).max())
    # the series needs its terms up to q^9 at |q| -> 1/8
    q = np.array([0.1249])
    exact = q - np.log1p(q)
    assert abs(phi_series(q, 9)[0] - exact[0]) / exact[0] < 2e-8
    assert abs(phi_series(q, 7)[0] - exact[0]) / exact[0] > 2e-8
