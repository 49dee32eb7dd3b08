"""Seeded synthetic scenes for the deconvolution workloads.

This module only *synthesises inputs*: true objects, point spread functions and
noisy detected images.  It holds none of the reconstruction arithmetic (no
Richardson-Lucy or SGP step, no KL value, no scaling, no projection); both the
CUDA path and the FP64 oracle receive the arrays produced here.

The paper's data (HST images of NGC7027/NGC6946/Crab, the RestoreTools AO PSF,
the LINC-NIRVANA PSFs, the Pleiades model) are not available, so the scenes
below stand in for them with the same structure: point sources with a large
dynamic range, smooth extended emission, band-limited diffraction PSFs, a
constant background and Poisson photon noise (Sect. 4.1 and 4.2 of the paper).

Every generator is driven by ``numpy.random.Generator(PCG64(seed))``; the same
seed gives bit-identical arrays on every machine.

Conventions
-----------
* Images are float64 arrays of shape (H, W) (or (p, H, W) for p views).
* PSFs are returned *centred*: the peak sits at pixel (H//2, W//2).  They are
  normalised to unit sum for convenience; the library and the oracle
  normalise again (the paper requires unit volume, Sect. 1 and 2.4).
* The detected image is ``g = Poisson(K * f + b)`` with a periodic blur on the
  scene grid, computed here by a numpy FFT (this is data synthesis, the
  forward model of the simulation, not the method).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ALLOWED_SIDES = tuple(sorted({2 ** a for a in range(4, 12)} | {3 * 2 ** a for a in range(3, 10)}))


def allowed_side(n: int) -> bool:
    return n in ALLOWED_SIDES


def next_allowed_side(n: int) -> int:
    for s in ALLOWED_SIDES:
        if s >= n:
            return s
    raise ValueError(f"no supported side >= {n} (max {ALLOWED_SIDES[-1]})")


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------- PSFs
def gaussian_psf(H: int, W: int, sigma: float) -> np.ndarray:
    y = np.arange(H) - H // 2
    x = np.arange(W) - W // 2
    r2 = y[:, None] ** 2 + x[None, :] ** 2
    k = np.exp(-0.5 * r2 / sigma ** 2)
    return k / k.sum()


def _disc(N: int, cy: float, cx: float, diameter: float) -> np.ndarray:
    """0/1 disc on an N x N grid; pixel centres inside the circle (wrap-around coordinates)."""
    y = np.arange(N, dtype=np.float64)
    y = np.where(y > N / 2, y - N, y)
    dy = y[:, None] - cy
    dx = y[None, :] - cx
    return ((dy ** 2 + dx ** 2) <= (diameter / 2.0) ** 2).astype(np.float64)


def _psf_from_pupil(pupil: np.ndarray) -> np.ndarray:
    amp = np.fft.fft2(pupil)
    k = np.abs(amp) ** 2
    k = np.fft.fftshift(k)          # peak to (N//2, N//2)
    return k / k.sum()


def airy_psf(N: int, diameter_frac: float = 1.0 / 8.0) -> np.ndarray:
    """|FFT of a circular pupil|^2, pupil diameter = diameter_frac * N (band-limited Airy pattern)."""
    return _psf_from_pupil(_disc(N, 0.0, 0.0, diameter_frac * N))


def two_pupil_psf(N: int, angle_deg: float, diameter_frac: float = 1.0 / 16.0,
                  separation_diameters: float = 3.0) -> np.ndarray:
    """Fizeau interferometer PSF: two circular pupils of diameter D = diameter_frac*N whose
    centres are separation_diameters*D apart along a baseline rotated by angle_deg."""
    D = diameter_frac * N
    half = 0.5 * separation_diameters * D
    a = math.radians(angle_deg)
    cy, cx = half * math.sin(a), half * math.cos(a)
    pupil = np.clip(_disc(N, cy, cx, D) + _disc(N, -cy, -cx, D), 0.0, 1.0)
    return _psf_from_pupil(pupil)


# --------------------------------------------------------------------------- objects
def star_field(rng: np.random.Generator, H: int, W: int, n: int, flux_lo: float = 1e3,
               flux_hi: float = 1e5, centre_sigma: float | None = None) -> np.ndarray:
    """Point sources on single pixels; fluxes log-uniform in [flux_lo, flux_hi].
    Positions uniform over the image, or Gaussian around the centre if centre_sigma is set."""
    f = np.zeros((H, W))
    if centre_sigma is None:
        ys = rng.integers(0, H, size=n)
        xs = rng.integers(0, W, size=n)
    else:
        ys = np.clip(np.rint(H / 2 + centre_sigma * rng.standard_normal(n)), 0, H - 1).astype(int)
        xs = np.clip(np.rint(W / 2 + centre_sigma * rng.standard_normal(n)), 0, W - 1).astype(int)
    fl = np.exp(rng.uniform(math.log(flux_lo), math.log(flux_hi), size=n))
    np.add.at(f, (ys, xs), fl)
    return f


def sersic_bn(n: float) -> float:
    """Ciotti & Bertin (1999) asymptotic expansion of the Sersic b_n constant."""
    return 2.0 * n - 1.0 / 3.0 + 4.0 / (405.0 * n) + 46.0 / (25515.0 * n * n)


def sersic_galaxy(rng: np.random.Generator, H: int, W: int, n_profiles: int = 5,
                  peak: float = 1e4) -> np.ndarray:
    """Sum of n_profiles Sersic profiles (index n ~ U[0.5, 4], effective radius ~ U[N/64, N/16],
    axis ratio ~ U[0.3, 1], position angle ~ U[0, pi), centres within N/8 of the image centre),
    rescaled to the given peak."""
    N = min(H, W)
    y = np.arange(H, dtype=np.float64)[:, None]
    x = np.arange(W, dtype=np.float64)[None, :]
    img = np.zeros((H, W))
    for _ in range(n_profiles):
        n = rng.uniform(0.5, 4.0)
        re = rng.uniform(N / 64.0, N / 16.0)
        q = rng.uniform(0.3, 1.0)
        th = rng.uniform(0.0, math.pi)
        cy = H / 2 + rng.uniform(-N / 8.0, N / 8.0)
        cx = W / 2 + rng.uniform(-N / 8.0, N / 8.0)
        dy, dx = y - cy, x - cx
        u = dx * math.cos(th) + dy * math.sin(th)
        v = -dx * math.sin(th) + dy * math.cos(th)
        r = np.sqrt(u * u + (v / q) ** 2)
        img += np.exp(-sersic_bn(n) * ((r / re) ** (1.0 / n) - 1.0))
    return img * (peak / img.max())


def gaussian_nebula(H: int, W: int, sigma: float, peak: float) -> np.ndarray:
    y = np.arange(H)[:, None] - H / 2
    x = np.arange(W)[None, :] - W / 2
    return peak * np.exp(-0.5 * (y * y + x * x) / sigma ** 2)


# --------------------------------------------------------------------------- forward model
def blur_periodic(f: np.ndarray, psf_centred: np.ndarray) -> np.ndarray:
    """Periodic blur used to *simulate* data (numpy FFT, float64)."""
    H, W = f.shape
    k0 = np.roll(psf_centred, (-(H // 2), -(W // 2)), axis=(0, 1))
    out = np.real(np.fft.ifft2(np.fft.fft2(k0) * np.fft.fft2(f)))
    return np.maximum(out, 0.0)


def poisson(rng: np.random.Generator, mean: np.ndarray) -> np.ndarray:
    return rng.poisson(np.maximum(mean, 0.0)).astype(np.float64)


# --------------------------------------------------------------------------- problems
@dataclass
class Scene:
    """One deconvolution problem: p views of an H x W object.

    psfs: (p, H, W) centred PSFs; g: (p, H, W) detected counts; b: (p,) constant backgrounds;
    mask: (H, W) uint8 M_S (1 on the detected-image pixels) or None for a periodic problem;
    f_true: (H, W) object used to simulate the data (on the same grid as g)."""
    psfs: np.ndarray
    g: np.ndarray
    b: np.ndarray
    f_true: np.ndarray
    mask: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def p(self) -> int:
        return self.g.shape[0]

    @property
    def shape(self) -> tuple[int, int]:
        return self.g.shape[1], self.g.shape[2]


def stars_scene(seed: int = 0, N: int = 256, n_stars: int = 50, sigma: float = 2.0,
                b: float = 10.0) -> Scene:
    """Single image: n_stars point stars at uniform pixels, fluxes log-uniform in [1e3, 1e5],
    zero sky; Gaussian PSF; constant background; Poisson noise (256 x 256 small case)."""
    rng = rng_for(seed)
    f = star_field(rng, N, N, n_stars)
    psf = gaussian_psf(N, N, sigma)
    g = poisson(rng, blur_periodic(f, psf) + b)
    return Scene(psfs=psf[None], g=g[None], b=np.array([b]), f_true=f,
                 meta=dict(kind="stars", N=N, seed=seed, sigma=sigma))


def galaxy_scene(seed: int = 0, N: int = 2048, n_stars: int = 500, b: float = 50.0,
                 diameter_frac: float = 1.0 / 8.0) -> Scene:
    """Single image: galaxy (5 Sersic profiles, peak 1e4) + n_stars log-uniform stars;
    Airy PSF from a circular pupil of diameter N/8; background 50; Poisson noise."""
    rng = rng_for(seed)
    f = sersic_galaxy(rng, N, N) + star_field(rng, N, N, n_stars)
    psf = airy_psf(N, diameter_frac)
    g = poisson(rng, blur_periodic(f, psf) + b)
    return Scene(psfs=psf[None], g=g[None], b=np.array([b]), f_true=f,
                 meta=dict(kind="galaxy", N=N, seed=seed))


def cluster_multiview_scene(seed: int = 0, N: int = 1024, p: int = 3, n_sources: int = 300,
                            b: float = 20.0) -> Scene:
    """p views of one object (star cluster of n_sources + diffuse Gaussian nebula), each blurred
    by a two-pupil interferometric PSF whose baseline is rotated by 180/p degrees per view."""
    rng = rng_for(seed)
    f = star_field(rng, N, N, n_sources, centre_sigma=N / 8.0) + gaussian_nebula(N, N, N / 10.0, 100.0)
    psfs = np.stack([two_pupil_psf(N, 180.0 * j / p) for j in range(p)])
    g = np.stack([poisson(rng, blur_periodic(f, psfs[j]) + b) for j in range(p)])
    return Scene(psfs=psfs, g=g, b=np.full(p, b), f_true=f,
                 meta=dict(kind="cluster", N=N, p=p, seed=seed))


def extended_side(n: int, sigma: float) -> int:
    """Side of the extended domain S-bar: smallest supported side >= n + 2*ceil(4 sigma)."""
    return next_allowed_side(n + 2 * int(math.ceil(4.0 * sigma)))


def boundary_scene(rng: np.random.Generator, n: int, sigma: float, b: float,
                   n_stars: int | None = None) -> Scene:
    """An n x n image cut from the centre of a 1.5n x 1.5n scene (so sources straddle the edge),
    Gaussian PSF of width sigma, background b, Poisson noise; embedded by zero padding in the
    extended domain S-bar (S centred) with the 0/1 mask M_S."""
    big = int(round(1.5 * n))
    ns = n_stars if n_stars is not None else max(20, (big * big) // 2000)
    scene = star_field(rng, big, big, ns) + sersic_galaxy(rng, big, big, n_profiles=2, peak=3e3)
    psf_big = gaussian_psf(big, big, sigma)
    mean_big = blur_periodic(scene, psf_big)
    o = (big - n) // 2
    g_cut = poisson(rng, mean_big[o:o + n, o:o + n] + b)
    Nb = extended_side(n, sigma)
    e = (Nb - n) // 2
    g = np.zeros((Nb, Nb))
    g[e:e + n, e:e + n] = g_cut
    mask = np.zeros((Nb, Nb), np.uint8)
    mask[e:e + n, e:e + n] = 1
    f_true = np.zeros((Nb, Nb))
    # object on S-bar: the part of the scene under the extended domain (for error measures)
    lo = o - e
    src = scene[max(lo, 0):lo + Nb, max(lo, 0):lo + Nb]
    d0 = max(-lo, 0)
    f_true[d0:d0 + src.shape[0], d0:d0 + src.shape[1]] = src
    psf = gaussian_psf(Nb, Nb, sigma)
    return Scene(psfs=psf[None], g=g[None], b=np.array([b]), f_true=f_true, mask=mask,
                 meta=dict(kind="boundary", n=n, N=Nb, sigma=sigma, offset=e))


def boundary_batch(seed: int = 0, count: int = 64,
                   sides: tuple[int, ...] = (128, 256, 384, 512, 768, 1024)) -> list[Scene]:
    """Batch of boundary problems: sides uniform over `sides`, sigma ~ U[1,4], b ~ U[5,50]."""
    rng = rng_for(seed)
    out = []
    for _ in range(count):
        n = int(rng.choice(sides))
        sigma = float(rng.uniform(1.0, 4.0))
        b = float(rng.uniform(5.0, 50.0))
        out.append(boundary_scene(rng, n, sigma, b))
    return out


def warmstart_scene(rng: np.random.Generator, N: int = 256) -> Scene:
    """Training/evaluation scene for the warm start: star-field or galaxy+stars object,
    Gaussian PSF with sigma ~ U[1,3], background 10 or 50, Poisson noise."""
    sigma = float(rng.uniform(1.0, 3.0))
    if rng.uniform() < 0.5:
        f = star_field(rng, N, N, int(rng.integers(20, 80)))
        b = 10.0
    else:
        f = sersic_galaxy(rng, N, N) + star_field(rng, N, N, int(rng.integers(20, 80)))
        b = 50.0
    psf = gaussian_psf(N, N, sigma)
    g = poisson(rng, blur_periodic(f, psf) + b)
    return Scene(psfs=psf[None], g=g[None], b=np.array([b]), f_true=f,
                 meta=dict(kind="warm", N=N, sigma=sigma))
