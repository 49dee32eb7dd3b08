"""FP64 CPU oracle of the RL / SGP deconvolution methods (Prato et al., Sect. 2 and 3).

TEST INFRASTRUCTURE ONLY.  Nothing in the CUDA product path imports, links or runs this file;
the test-suite, the smoke check and the benchmark's CPU-baseline leg are its only users.

Plain, slow, obviously correct numpy in float64.  The periodic convolution and correlation use
numpy's FFT as a library primitive; everything else follows the paper's definitions and
algorithm steps in the paper's order and notation:

  A_j f      = M_S . (K_j * (M_R f))                 Sect. 2.4, Eq. (projection)
  A_j^T y    = M_R . (K_j (x) (M_S y))               Sect. 2.4, Eq. (backprojection)
  J_0        = sum_j sum_m g ln(g/(A f+b)) + A f + b - g   Sect. 1 Eq. (KL), Sect. 2.3 Eq. (multipleKL)
  grad J_0   = sum_j A_j^T 1 - A_j^T (g_j/(A_j f + b_j))   Eq. (KLgrad), (multiplegradient), (gradientboundary)
  RL step    = (M_R/alpha) . f . sum_j A_j^T r_j      Eq. (RL), (multipleRL), (boundaryRL)
  SGP        = Algorithm 1 with scaled BB1/BB2 (Eq. BB1, BB2), safeguards and alternation
               (Eq. alphadef), scaling (Eq. Dk / Dkbound), parameters of Sect. 3.2
  OSEM       = Algorithm 2, Eq. (OSEMstep) / (boundaryOSEM)
  mosaic     = Sect. 4, second experiment (Table 2, Table 6): overlapping sub-domains, each
               reconstructed with boundary-effect correction on a zero-padded array, the
               non-overlapping central parts put together
  stop rules = Sect. 3.3 (fixed, Eq. convergence, min. reconstruction error, Eq. discrepancy)

Readings of places where the paper is silent or garbled (all stated again in the design notes):
  * PSF origin: the PSF is given centred (peak at (H//2, W//2)) and rolled to (0, 0); it is
    normalised to unit sum over the (extended) domain; tiny negative round-off is clamped to 0.
  * alpha_j(n) = sum_m K_j(m-n) M_S(m) (the printed formula carries a stray factor g(m); without
    it A_j^T 1 = M_R alpha_j, which the gradient Eq. (gradientboundary) needs, and alpha = p when
    the masks are all ones, so boundary RL reduces to multiple RL).
  * multi-image periodic scaling: D = clip(f, L1, L2)/p (the masks-all-ones case of Eq. Dkbound).
  * ratio g/(A f + b) is 0 where A f + b = 0; the KL term is +inf where A f + b = 0 < g.
  * BB sums use D_k of the new iterate f^(k) and run over the pixels where D_k > 0.
  * k = 0 uses alpha_0; for k = 1..20 alpha_k is the windowed minimum of Eq. (alphadef) and tau is
    not updated; the alternation test runs from k = 21 with tau = tau_1.  "10 alpha_{k-1}" uses
    the alpha actually taken at k-1.
  * Armijo loop: at most 30 reductions of lambda (error beyond).
  * L1/L2: one RL step from f^(0) in the active mode; y_min/y_max over strictly positive pixels;
    the test is "< 50" exactly.
  * constant start: c = mean over views of (sum_S g_j - sum_S b_j)/|S|, put on R (on the whole
    domain without a boundary); if c <= 0 then c = max(mean g, 1e-3).
  * discrepancy D = 2 J_0/(p |S|); stop at the first k with D <= eta and return f^(k).
  * flux-constrained projection (the paper defers it to Bonettini et al.): the D^-1-weighted
    projection onto {y >= 0, sum y = c}, y_i = max(0, x_i - mu D_i), mu solved exactly from the
    sorted breakpoints.
  * regularised SGP (Sect. 5 names the extension and the split-gradient scaling of Lanteri et al.,
    no regulariser): J_0 + beta/2 ||f||^2 (Tikhonov); split grad = V - U with V = sum_j A_j^T 1 +
    beta f, U = sum_j A_j^T r_j, scaling D = clip(f)/V_bar with V_bar = sum_j A_j^T 1 + beta clip(f);
    the Armijo test and the convergence rule use J_0 + R, the discrepancy rule J_0 alone.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "prepare_psf", "set_fft_workers", "set_fft_single_precision", "conv_periodic", "corr_periodic", "Problem", "SGPParams", "StopRule",
    "sgp", "rl", "osem", "bb_steplengths", "choose_alpha", "adaptive_bounds",
    "flux_projection", "kl_terms", "mosaic_axis", "mosaic_split", "mosaic_stitch", "mosaic",
]


# ----------------------------------------------------------------------------- PSF
def prepare_psf(psf, origin: str = "center") -> np.ndarray:
    """Unit-volume PSF with its origin at pixel (0, 0) (Sect. 1; Sect. 2.4: normalised over S-bar).

    psf: (H, W) samples; with origin='center' the PSF origin is at (H//2, W//2)."""
    K = np.array(psf, dtype=np.float64, copy=True)
    if K.ndim != 2:
        raise ValueError("PSF must be 2-D")
    mx = K.max()
    if not np.isfinite(K).all() or mx <= 0.0:
        raise ValueError("PSF must be finite with a positive maximum")
    if K.min() < -1e-6 * mx:
        raise ValueError("PSF has significantly negative samples")
    K = np.maximum(K, 0.0)
    s = K.sum()
    K /= s
    if origin == "center":
        H, W = K.shape
        K = np.roll(K, (-(H // 2), -(W // 2)), axis=(0, 1))
    elif origin != "corner":
        raise ValueError("origin must be 'center' or 'corner'")
    return K


_FFT_WORKERS = None   # None: numpy.fft (one thread); n: scipy.fft with n worker threads
_FFT_SINGLE = False   # True: the transforms in single precision (inputs rounded to float32)


def set_fft_workers(n: int | None) -> None:
    """Run the FFT primitive of the two convolutions below on n host threads (scipy.fft, the same
    pocketfft transform as numpy.fft, split over its rows and columns), or on one thread through
    numpy.fft (None, the default).  Only the library primitive changes; every other step of the
    oracle stays single-threaded numpy."""
    global _FFT_WORKERS
    _FFT_WORKERS = None if n is None or n <= 1 else int(n)


def set_fft_single_precision(on: bool) -> None:
    """Evaluate the two convolutions below with single-precision transforms (inputs rounded to
    float32, numpy.fft in complex64, results returned as float64), or in double precision (the
    default).  This models the rounding of FP32 transforms alone, for bounding how far an FP32
    implementation of the method can drift from the FP64 oracle; every other step stays FP64."""
    global _FFT_SINGLE
    _FFT_SINGLE = bool(on)


def _fft2(x):
    if _FFT_SINGLE:
        return np.fft.fft2(np.asarray(x).astype(np.complex64))
    if _FFT_WORKERS is None:
        return np.fft.fft2(x)
    import scipy.fft
    return scipy.fft.fft2(x, workers=_FFT_WORKERS)


def _ifft2(x):
    if _FFT_SINGLE:
        return np.fft.ifft2(np.asarray(x).astype(np.complex64))
    if _FFT_WORKERS is None:
        return np.fft.ifft2(x)
    import scipy.fft
    return scipy.fft.ifft2(x, workers=_FFT_WORKERS)


def conv_periodic(f: np.ndarray, K: np.ndarray) -> np.ndarray:
    """(K * f)(m) = sum_n K(m - n) f(n), indices modulo the array shape (FFT as a primitive)."""
    return np.real(_ifft2(_fft2(K) * _fft2(f))).astype(np.float64)


def corr_periodic(y: np.ndarray, K: np.ndarray) -> np.ndarray:
    """(K (x) y)(n) = sum_m K(m - n) y(m): the transpose of conv_periodic for real K."""
    return np.real(_ifft2(np.conj(_fft2(K)) * _fft2(y))).astype(np.float64)


def kl_terms(g: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Pixel terms g ln(g/u) + u - g of Eq. (KL) with u = A f + b, 0 ln 0 = 0, +inf if u = 0 < g."""
    out = np.array(u - g, dtype=np.float64)
    pos = g > 0
    with np.errstate(divide="ignore", invalid="ignore"):
        lg = np.where(pos & (u > 0), g * np.log(np.where(pos, g, 1.0) / np.where(u > 0, u, 1.0)), 0.0)
    out = out + lg
    out[pos & (u <= 0)] = np.inf
    return out


# ----------------------------------------------------------------------------- problem
class Problem:
    """p detected images g_j of one object f, PSFs K_j, backgrounds b_j, optional boundary mask.

    psfs: (p, H, W); g: (p, H, W); b: (p,) constants or (p, H, W) arrays;
    mask_S: None (periodic problem, Sect. 2.2-2.3) or (H, W) 0/1 array M_S on the extended
    domain S-bar (Sect. 2.4); sigma_R: threshold of Eq. (Rdef)."""

    def __init__(self, psfs, g, b, mask_S=None, sigma_R: float = 1e-2, origin: str = "center"):
        psfs = np.asarray(psfs, np.float64)
        g = np.asarray(g, np.float64)
        if psfs.ndim == 2:
            psfs = psfs[None]
        if g.ndim == 2:
            g = g[None]
        self.p, self.H, self.W = g.shape
        if psfs.shape != g.shape:
            raise ValueError("psfs and g must have the same (p, H, W) shape")
        self.K = [prepare_psf(psfs[j], origin) for j in range(self.p)]
        b = np.asarray(b, np.float64)
        if b.ndim <= 1:
            b = np.broadcast_to(b.reshape(-1, 1, 1) if b.ndim == 1 else b, (self.p, self.H, self.W))
        self.boundary = mask_S is not None
        if self.boundary:
            self.MS = (np.asarray(mask_S) != 0).astype(np.float64)
        else:
            self.MS = np.ones((self.H, self.W))
        # data are merged into S-bar by zero padding (Sect. 2.4)
        self.g = g * self.MS
        self.b = np.array(b) * self.MS
        if self.boundary:
            # alpha_j(n) = sum_m K_j(m - n) M_S(m) (reading: no factor g), Eq. (Rdef)
            self.alpha_j = [corr_periodic(self.MS, K) for K in self.K]
            R = np.ones((self.H, self.W), bool)
            for a in self.alpha_j:
                R &= a >= sigma_R
            self.MR = R.astype(np.float64)
        else:
            self.alpha_j = [np.ones((self.H, self.W)) for _ in self.K]
            self.MR = np.ones((self.H, self.W))
        alpha = np.sum(self.alpha_j, axis=0)
        # M_R / alpha, zero outside R (Eq. boundaryRL: "the quotient being zero outside R")
        self.w = np.where(self.MR > 0, 1.0 / np.where(self.MR > 0, alpha, 1.0), 0.0)
        self.alpha = alpha
        self.nS = float(self.MS.sum())

    # operators, Eq. (projection) and (backprojection); periodic problems have M_S = M_R = 1
    def A(self, j: int, f: np.ndarray) -> np.ndarray:
        return self.MS * conv_periodic(self.MR * f, self.K[j])

    def AT(self, j: int, y: np.ndarray) -> np.ndarray:
        return self.MR * corr_periodic(self.MS * y, self.K[j])

    def ratio(self, j: int, Af: np.ndarray) -> np.ndarray:
        u = Af + self.b[j]
        with np.errstate(divide="ignore", invalid="ignore"):
            return np.where(u > 0, self.g[j] / np.where(u > 0, u, 1.0), 0.0) * self.MS

    def kl(self, f: np.ndarray, Afs=None) -> float:
        """J_0(f; g), Eq. (KL) / (multipleKL); sum over m in S."""
        tot = 0.0
        for j in range(self.p):
            Af = self.A(j, f) if Afs is None else Afs[j]
            t = kl_terms(self.g[j], Af + self.b[j])
            tot += float(np.sum(t[self.MS > 0]))
        return tot

    def grad(self, f: np.ndarray) -> np.ndarray:
        """Eq. (KLgrad) / (multiplegradient) / (gradientboundary)."""
        out = np.zeros((self.H, self.W))
        ones = np.ones((self.H, self.W))
        for j in range(self.p):
            out += self.AT(j, ones) - self.AT(j, self.ratio(j, self.A(j, f)))
        return out

    def rl_step(self, f: np.ndarray) -> np.ndarray:
        """One (multiple / boundary) RL iteration, Eq. (RL), (multipleRL), (boundaryRL)."""
        s = np.zeros((self.H, self.W))
        for j in range(self.p):
            s += self.AT(j, self.ratio(j, self.A(j, f)))
        return self.w * f * s

    def discrepancy(self, J: float) -> float:
        """Eq. (discrepancy): 2 J_0 / (p N^2), N^2 -> |S|."""
        return 2.0 * J / (self.p * self.nS)

    def initial(self, mode: str = "constant", f_user=None) -> np.ndarray:
        """Starting points of Sect. 3.1."""
        if mode == "zero":
            return np.zeros((self.H, self.W))
        if mode == "data":
            return self.g[0].copy()
        if mode == "user":
            return np.maximum(np.asarray(f_user, np.float64), 0.0) * self.MR
        if mode != "constant":
            raise ValueError(mode)
        fl = [(self.g[j][self.MS > 0].sum() - self.b[j][self.MS > 0].sum()) / self.nS
              for j in range(self.p)]
        c = float(np.mean(fl))
        if c <= 0.0:
            c = max(float(np.mean([self.g[j][self.MS > 0].mean() for j in range(self.p)])), 1e-3)
        return c * self.MR


# ----------------------------------------------------------------------------- parameters
@dataclass
class SGPParams:
    """Sect. 3.2 values."""
    beta: float = 1e-4
    theta: float = 0.4
    alpha0: float = 1.3
    tau1: float = 0.5
    alpha_min: float = 1e-5
    alpha_max: float = 1e5
    M_alpha: int = 3
    warmup_iters: int = 20
    adaptive_L: bool = True
    L1: float = 1e-10
    L2: float = 1e10
    max_backtracks: int = 30
    flux: float | None = None      # None: non-negativity only; else the flux constraint sum f = flux
    reg_beta: float = 0.0          # > 0: minimise J_0 + reg_beta/2 ||f||^2 (Tikhonov, SGM scaling)


@dataclass
class StopRule:
    """Sect. 3.3: kind in {'fixed', 'convergence', 'discrepancy', 'min_error', 'landed'}.

    'landed' (SGP only; a reading, not in the paper): the discrepancy stop with the last step
    shortened so that the final discrepancy is eta (1 - tol/2), found by bisection on the step
    length; tol <= 0 means 1e-5."""
    kind: str = "fixed"
    max_iter: int = 100
    tol: float = 1e-4
    eta: float = 1.0
    f_true: np.ndarray | None = None


def adaptive_bounds(y: np.ndarray) -> tuple[float, float]:
    """(L1, L2) from one RL step y (Sect. 3.2): over the strictly positive values of y."""
    pos = y[y > 0]
    if pos.size == 0:
        raise ValueError("the RL step has no positive pixel")
    ymin, ymax = float(pos.min()), float(pos.max())
    if ymax / ymin < 50.0:
        return ymin / 10.0, ymax * 10.0
    return ymin, ymax


def bb_steplengths(s: np.ndarray, z: np.ndarray, D: np.ndarray) -> tuple[float, float, float, float]:
    """Numerators and denominators of the scaled BB rules, Eq. (BB1)-(BB2), over pixels D > 0:
    (s^T D^-1 D^-1 s, s^T D^-1 z, s^T D z, z^T D D z)."""
    m = D > 0
    s, z, D = s[m], z[m], D[m]
    return (float(np.sum(s * s / (D * D))), float(np.sum(s * z / D)),
            float(np.sum(s * z * D)), float(np.sum(z * z * D * D)))


@dataclass
class AlphaState:
    alpha_prev: float
    tau: float
    hist: list = field(default_factory=list)   # alpha^(2)_j values, j = 1..k


def choose_alpha(k: int, sums, st: AlphaState, P: SGPParams) -> tuple[float, int]:
    """Step 1 of Algorithm 1 for k >= 1: safeguarded BB values and the alternation of
    Eq. (alphadef); returns (alpha_k, branch) with branch 2 = windowed BB2, 1 = BB1."""
    n1, d1, n2, d2 = sums
    if d1 <= 0.0:
        a1 = min(10.0 * st.alpha_prev, P.alpha_max)
    else:
        a1 = min(P.alpha_max, max(P.alpha_min, n1 / d1))
    if n2 <= 0.0:                       # s^T D z <= 0
        a2 = min(10.0 * st.alpha_prev, P.alpha_max)
    else:
        a2 = min(P.alpha_max, max(P.alpha_min, n2 / d2))
    st.hist.append(a2)
    window = st.hist[-P.M_alpha:]       # j = max(1, k+1-M_alpha), ..., k
    if k <= P.warmup_iters:
        alpha, branch = min(window), 2
    elif a2 / a1 <= st.tau:
        alpha, branch = min(window), 2
        st.tau *= 0.9
    else:
        alpha, branch = a1, 1
        st.tau *= 1.1
    st.alpha_prev = alpha
    return alpha, branch


def flux_projection(x: np.ndarray, D: np.ndarray, c: float) -> np.ndarray:
    """argmin_y sum_i (y_i - x_i)^2 / D_i subject to y >= 0, sum y = c (pixels with D_i = 0 are
    kept at x_i and count toward the sum).  KKT: y_i = max(0, x_i - mu D_i), with mu the root of
    the non-increasing piecewise-linear phi(mu) = sum_i max(0, x_i - mu D_i) - c', found exactly
    from the sorted breakpoints t_i = x_i / D_i."""
    x = np.asarray(x, np.float64)
    D = np.asarray(D, np.float64)
    act = D > 0
    fixed_sum = float(x[~act].sum())
    cp = c - fixed_sum
    xa, Da = x[act], D[act]
    if cp <= 0.0 or xa.size == 0:
        y = x.copy()
        y[act] = 0.0
        return y
    t = xa / Da
    order = np.argsort(-t)                     # decreasing breakpoints
    ts, xs, Ds = t[order], xa[order], Da[order]
    # with the first n breakpoints active: phi(mu) = X_n - mu S_n - cp, valid for mu in [t_{n+1}, t_n]
    Xn = np.cumsum(xs)
    Sn = np.cumsum(Ds)
    mu = None
    for n in range(1, xs.size + 1):
        m = (Xn[n - 1] - cp) / Sn[n - 1]
        lo = ts[n] if n < xs.size else -np.inf
        if lo <= m <= ts[n - 1]:
            mu = m
            break
    if mu is None:                             # numerically at a breakpoint
        mu = float(ts[-1])
    y = x.copy()
    y[act] = np.maximum(0.0, xa - mu * Da)
    return y


# ----------------------------------------------------------------------------- regularisation (Sect. 5)
def reg_value(f: np.ndarray, beta: float) -> float:
    """Tikhonov term J_R = beta/2 sum f^2 (reading of the regularised SGP of Sect. 5: the paper names
    no regularisation function; this is the simplest one whose split-gradient scaling is explicit)."""
    return 0.5 * beta * float(np.sum(f * f))


def sgm_split(prob: "Problem", f: np.ndarray, beta: float):
    """Split-gradient decomposition grad J = V - U with V, U >= 0 for f >= 0 (Lanteri et al., cited in
    Sect. 5): for J_0, V_0 = sum_j A_j^T 1 and U_0 = sum_j A_j^T (g_j/(A_j f + b_j)) (Eq. KLgrad); for
    beta/2 ||f||^2, V_R = beta f and U_R = 0.  Returns (V, U)."""
    V = np.zeros((prob.H, prob.W))
    U = np.zeros((prob.H, prob.W))
    ones = np.ones((prob.H, prob.W))
    for j in range(prob.p):
        V += prob.AT(j, ones)
        U += prob.AT(j, prob.ratio(j, prob.A(j, f)))
    return V + beta * f, U


def sgm_scaling(prob: "Problem", f: np.ndarray, L1: float, L2: float, beta: float) -> np.ndarray:
    """SGP scaling built from the split: D = c / V_bar with c = clip(f, L1, L2) and
    V_bar = (sum_j A_j^T 1) + beta c, i.e. D = w c / (1 + beta w c) with w = M_R/alpha (1/p periodic),
    0 outside R.  With beta = 0 it is w clip(f, L1, L2), the scaling of Eq. (Dk)/(Dkbound)."""
    c = np.minimum(L2, np.maximum(L1, f))
    if beta == 0.0:
        return prob.w * c
    return prob.w * c / (1.0 + beta * prob.w * c)


# ----------------------------------------------------------------------------- SGP
@dataclass
class Result:
    f: np.ndarray
    iters: int
    J: float
    trace: list
    status: str = "ok"
    L1: float = 0.0
    L2: float = 0.0


def _stop_check(rule: StopRule, k: int, J_old: float, J_new: float, D_new: float) -> bool:
    if rule.kind == "convergence":
        return abs(J_new - J_old) <= rule.tol * J_old
    if rule.kind in ("discrepancy", "landed"):
        return D_new <= rule.eta
    return False


def _land(prob: Problem, f, d, J, lam, Jn, rule: StopRule):
    """Shorten an accepted step f + lam d whose discrepancy is below eta: the step length in
    (0, lam] where D = eta (1 - tol/2), by bisection (J is convex along the step, J(0) above the
    target, J(lam) below).  A(f + t d) = A f + t A d by linearity.  Returns (t, J(t), f + t d)."""
    tol = rule.tol if rule.tol > 0 else 1e-5
    Jt = rule.eta * (1.0 - 0.5 * tol) / prob.discrepancy(1.0)
    if not (Jn < Jt < J):
        return lam, Jn, f + lam * d
    Afs = [prob.A(j, f) for j in range(prob.p)]
    Ads = [prob.A(j, d) for j in range(prob.p)]
    Jat = lambda t: prob.kl(f + t * d, [Afs[j] + t * Ads[j] for j in range(prob.p)])
    lo, hi = 0.0, lam
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if Jat(mid) > Jt:
            lo = mid
        else:
            hi = mid
    return hi, Jat(hi), f + hi * d


def _rel_err(f, ft):
    return float(np.linalg.norm(f - ft) / np.linalg.norm(ft))


def sgp(prob: Problem, f0: np.ndarray | None = None, P: SGPParams | None = None,
        stop: StopRule | None = None) -> Result:
    """Algorithm 1 (monotone SGP) for min_{f >= 0} J_0(f; g) on the given problem."""
    P = P or SGPParams()
    stop = stop or StopRule()
    f = prob.initial("constant") if f0 is None else np.array(f0, np.float64)
    if P.flux is not None:
        tot = f.sum()
        f = f * (P.flux / tot) if tot > 0 else f
    if P.adaptive_L:
        L1, L2 = adaptive_bounds(prob.rl_step(f))
    else:
        L1, L2 = P.L1, P.L2
    Afs = [prob.A(j, f) for j in range(prob.p)]
    beta_r = P.reg_beta
    J = prob.kl(f, Afs)
    R = reg_value(f, beta_r)               # the objective is J + R (R = 0 without regularisation)
    trace = []
    st = AlphaState(alpha_prev=P.alpha0, tau=P.tau1)
    g_prev = f_prev = None
    rho_prev = _rel_err(f, stop.f_true) if stop.kind == "min_error" else None
    if stop.kind in ("discrepancy", "landed") and prob.discrepancy(J) <= stop.eta:
        return Result(f, 0, J, trace, L1=L1, L2=L2)
    k = 0
    while k < stop.max_iter:
        grad = prob.grad(f) + beta_r * f
        # step 1: scaling Eq. (Dk)/(Dkbound) (with a regulariser: the split-gradient scaling) and step length
        D = sgm_scaling(prob, f, L1, L2, beta_r)
        if k == 0:
            alpha, branch = P.alpha0, 0
            st.alpha_prev = alpha
        else:
            alpha, branch = choose_alpha(k, bb_steplengths(f - f_prev, grad - g_prev, D), st, P)
        # step 2: projection, Eq. (diry)
        x = f - alpha * D * grad
        y = np.maximum(x, 0.0) if P.flux is None else flux_projection(x, D, P.flux)
        # step 3: descent direction
        d = y - f
        gTd = float(np.sum(grad * d))
        # steps 4-5: Armijo backtracking
        lam, nb = 1.0, 0
        while True:
            fl = f + lam * d
            Afl = [prob.A(j, fl) for j in range(prob.p)]
            Jn = prob.kl(fl, Afl)
            Rn = reg_value(fl, beta_r)
            if Jn + Rn <= J + R + P.beta * lam * gTd:
                break
            nb += 1
            if nb > P.max_backtracks:
                return Result(f, k, J, trace, status="linesearch", L1=L1, L2=L2)
            lam *= P.theta
        if stop.kind == "landed" and prob.discrepancy(Jn) <= stop.eta:
            lam, Jn, fl = _land(prob, f, d, J, lam, Jn, stop)
            Rn = reg_value(fl, beta_r)
        # step 6
        f_prev, g_prev = f, grad
        f = fl
        J0_old, J_old = J, J + R             # J_0 and the objective J_0 + R before the step
        J, R = Jn, Rn
        k += 1
        trace.append(dict(k=k, J=J, D=prob.discrepancy(J), alpha=alpha, lam=lam,
                          backtracks=nb, branch=branch, gTd=gTd, R=R))
        if stop.kind == "min_error":
            rho = _rel_err(f, stop.f_true)
            trace[-1]["rho"] = rho
            if rho > rho_prev:
                return Result(f_prev, k - 1, J0_old, trace, L1=L1, L2=L2)
            rho_prev = rho
        if _stop_check(stop, k, J_old, J + R, prob.discrepancy(J)):
            break
    return Result(f, k, J, trace, L1=L1, L2=L2)


def rl(prob: Problem, f0: np.ndarray | None = None, stop: StopRule | None = None) -> Result:
    """Richardson-Lucy iterations (single, multiple or boundary form)."""
    stop = stop or StopRule()
    f = prob.initial("constant") if f0 is None else np.array(f0, np.float64)
    J = prob.kl(f)
    trace = []
    rho_prev = _rel_err(f, stop.f_true) if stop.kind == "min_error" else None
    if stop.kind == "discrepancy" and prob.discrepancy(J) <= stop.eta:
        return Result(f, 0, J, trace)
    k = 0
    while k < stop.max_iter:
        f_prev = f
        f = prob.rl_step(f)
        J_old, J = J, prob.kl(f)
        k += 1
        trace.append(dict(k=k, J=J, D=prob.discrepancy(J)))
        if stop.kind == "min_error":
            rho = _rel_err(f, stop.f_true)
            trace[-1]["rho"] = rho
            if rho > rho_prev:
                return Result(f_prev, k - 1, J_old, trace)
            rho_prev = rho
        if _stop_check(stop, k, J_old, J, prob.discrepancy(J)):
            break
    return Result(f, k, J, trace)


def osem(prob: Problem, f0: np.ndarray | None = None, n_iter: int = 10) -> Result:
    """Algorithm 2 (OSEM) with Eq. (OSEMstep), or Eq. (boundaryOSEM) with a boundary mask."""
    f = prob.initial("constant") if f0 is None else np.array(f0, np.float64)
    for _ in range(n_iter):
        h = f
        for j in range(prob.p):
            v = prob.AT(j, prob.ratio(j, prob.A(j, h)))
            if prob.boundary:
                aj = prob.alpha_j[j]
                wj = np.where(prob.MR > 0, 1.0 / np.where(prob.MR > 0, aj, 1.0), 0.0)
                h = wj * h * v
            else:
                h = h * v
        f = h
    return Result(f, n_iter, prob.kl(f), [])


# ----------------------------------------------------------------------------- mosaic
def mosaic_axis(N: int, n: int, s: int) -> list[tuple[int, int, int, int]]:
    """One axis of the mosaic of Sect. 4 (second experiment): N pixels covered by n partially
    overlapping sub-domains of s pixels and cut into n non-overlapping pieces.

    Reading (the paper gives only the 256 -> 4 x 160^2 -> 4 x 128^2 example): sub-domain k starts
    at floor(k (N - s) / (n - 1)) (0 for n = 1), so the first starts at 0 and the last ends at N;
    piece k is [floor(k N / n), floor((k + 1) N / n)) and must lie inside sub-domain k.
    Returns (sub-domain start, end, piece start, end) for k = 0..n-1."""
    if n < 1 or s < 1 or s > N:
        raise ValueError("need 1 <= s <= N and n >= 1")
    out = []
    for k in range(n):
        w0 = 0 if n == 1 else (k * (N - s)) // (n - 1)
        c0, c1 = (k * N) // n, ((k + 1) * N) // n
        if c0 < w0 or c1 > w0 + s:
            raise ValueError("piece %d [%d, %d) is not inside sub-domain [%d, %d)" % (k, c0, c1, w0, w0 + s))
        out.append((w0, w0 + s, c0, c1))
    return out


def mosaic_split(g: np.ndarray, n, sub, ext):
    """Sub-images of g (p, H, W) merged by zero padding into ext-sized arrays, the sub-image
    centred (offset floor((ext - sub)/2)), with the masks M_S (1 on the sub-image).
    Returns g_tiles (ny*nx, p, EH, EW) and masks (ny*nx, EH, EW), tiles in row-major order."""
    g = np.asarray(g, np.float64)
    if g.ndim == 2:
        g = g[None]
    p, H, W = g.shape
    ay, ax = mosaic_axis(H, n[0], sub[0]), mosaic_axis(W, n[1], sub[1])
    ey, ex = (ext[0] - sub[0]) // 2, (ext[1] - sub[1]) // 2
    tiles, masks = [], []
    for (y0, y1, _, _) in ay:
        for (x0, x1, _, _) in ax:
            t = np.zeros((p, ext[0], ext[1]))
            t[:, ey:ey + sub[0], ex:ex + sub[1]] = g[:, y0:y1, x0:x1]
            m = np.zeros((ext[0], ext[1]), np.uint8)
            m[ey:ey + sub[0], ex:ex + sub[1]] = 1
            tiles.append(t)
            masks.append(m)
    return np.stack(tiles), np.stack(masks)


def mosaic_stitch(recs: np.ndarray, shape, n, sub, ext) -> np.ndarray:
    """The mosaic: piece (ky, kx) of the H x W image taken from reconstruction ky*nx + kx."""
    H, W = shape
    ay, ax = mosaic_axis(H, n[0], sub[0]), mosaic_axis(W, n[1], sub[1])
    ey, ex = (ext[0] - sub[0]) // 2, (ext[1] - sub[1]) // 2
    out = np.zeros((H, W))
    for ky, (y0, _, c0, c1) in enumerate(ay):
        for kx, (x0, _, d0, d1) in enumerate(ax):
            r = recs[ky * len(ax) + kx]
            out[c0:c1, d0:d1] = r[ey + c0 - y0:ey + c1 - y0, ex + d0 - x0:ex + d1 - x0]
    return out


def mosaic(psfs_ext, g, b, n=(2, 2), sub=(160, 160), ext=(256, 256), method: str = "sgp",
           n_iter: int = 50, sigma_R: float = 1e-2) -> np.ndarray:
    """Boundary-corrected reconstruction of g (p, H, W) as a mosaic (Sect. 4, Table 2 / Table 6):
    every sub-domain is reconstructed on its own zero-padded ext-sized array with the
    boundary-effect correction of Sect. 2.4 (PSFs psfs_ext given on that array, centred), by
    n_iter iterations of SGP, RL or OSEM; the pieces are put together."""
    g = np.asarray(g, np.float64)
    if g.ndim == 2:
        g = g[None]
    tiles, masks = mosaic_split(g, n, sub, ext)
    recs = []
    for t, m in zip(tiles, masks):
        prob = Problem(psfs_ext, t, b, mask_S=m, sigma_R=sigma_R)
        if method == "sgp":
            recs.append(sgp(prob, stop=StopRule("fixed", max_iter=n_iter)).f)
        elif method == "rl":
            recs.append(rl(prob, stop=StopRule("fixed", max_iter=n_iter)).f)
        else:
            recs.append(osem(prob, n_iter=n_iter).f)
    return mosaic_stitch(np.stack(recs), g.shape[-2:], n, sub, ext)
