"""Seeded synthetic inputs for the porous-cavity and porous-channel workloads.

This module holds only input generation (random fields, parameter draws and
named workload settings).  It contains none of the lattice Boltzmann
arithmetic, imports nothing else from this package, and is the one module
shared by the CUDA path's callers and by the CPU oracle's callers.

Workloads (the paper's own configurations are synthetic by nature; no public
dataset is involved):
  * natural convection in a square porous cavity (Sec. 3.2, Table 1);
  * spatially varying porosity eps(x) = 0.3 + 0.6 Phi(g(x)), g a zero-mean,
    unit-variance Gaussian random field with Gaussian covariance
    exp(-r^2 / (2 l^2)), l = 32 cells, Phi the standard normal CDF;
  * body-force-driven porous channel (Brinkman profile) and the mixed
    convection channel of Sec. 3.1;
  * a seeded batch of independent cavities with log-uniform sizes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

PHI_SEED = 20211012


def gaussian_random_field(nx: int, ny: int, ell: float = 32.0, seed: int = PHI_SEED) -> np.ndarray:
    """Periodic Gaussian random field on an (ny, nx) grid.

    Seeded N(0, 1) white noise is filtered in Fourier space by
    exp(-ell^2 |k|^2 / 4), the square root of the spectrum of the covariance
    exp(-r^2 / (2 ell^2)), then shifted and scaled to zero mean and unit
    variance.  Returns float64."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((ny, nx))
    kx = 2.0 * np.pi * np.fft.rfftfreq(nx)
    ky = 2.0 * np.pi * np.fft.fftfreq(ny)
    k2 = ky[:, None] ** 2 + kx[None, :] ** 2
    filt = np.exp(-0.25 * ell * ell * k2)
    g = np.fft.irfft2(np.fft.rfft2(w) * filt, s=(ny, nx))
    g -= g.mean()
    sd = g.std()
    if sd > 0:
        g /= sd
    return np.ascontiguousarray(g)


def _normal_cdf(x: np.ndarray) -> np.ndarray:
    try:
        from scipy.special import ndtr
        return ndtr(x)
    except Exception:  # pragma: no cover - scipy is present on both machines
        v = np.vectorize(lambda t: 0.5 * math.erfc(-t / math.sqrt(2.0)))
        return v(x)


def porosity_field(nx: int, ny: int, seed: int = PHI_SEED, ell: float = 32.0,
                   lo: float = 0.3, span: float = 0.6) -> np.ndarray:
    """eps(x) = lo + span * Phi(g(x)) with g from gaussian_random_field."""
    g = gaussian_random_field(nx, ny, ell, seed)
    return np.ascontiguousarray(lo + span * _normal_cdf(g))


def smooth_fields(nx: int, ny: int, seed: int, amp_u: float = 0.02, amp_rho: float = 0.01,
                  amp_T: float = 0.2):
    """Smooth random (rho, ux, uy, T) fields for non-trivial initial states:
    a few seeded low Fourier modes, periodic on the grid."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    out = []
    for amp, base in ((amp_rho, 1.0), (amp_u, 0.0), (amp_u, 0.0), (amp_T, 0.5)):
        fld = np.full((ny, nx), base)
        for _ in range(3):
            kx, ky = rng.integers(0, 3), rng.integers(0, 3)
            ph = rng.uniform(0, 2 * np.pi)
            fld += amp / 3.0 * np.cos(2 * np.pi * (kx * x / nx + ky * y / ny) + ph)
        out.append(np.ascontiguousarray(fld))
    return tuple(out)


@dataclass(frozen=True)
class CavityCase:
    """One natural-convection cavity: grid and dimensionless groups."""
    nx: int
    ny: int
    Ra: float
    Da: float
    Pr: float
    phi: float          # uniform porosity, or the mean for a random field
    sigma: float
    J: float = 1.0
    Gamma: float = 1.0


# Named workloads: uniform-porosity cavity of Table 1 at 64^2, the seeded
# random-porosity cavities at 4096^2 and 8192^2, and the Brinkman channel.
CAVITY_64 = CavityCase(64, 64, Ra=1e4, Da=1e-2, Pr=1.0, phi=0.6, sigma=1.0)
CAVITY_4096 = CavityCase(4096, 4096, Ra=1e6, Da=1e-3, Pr=0.71, phi=float("nan"), sigma=1.0)
CAVITY_8192 = CavityCase(8192, 8192, Ra=1e6, Da=1e-3, Pr=0.71, phi=float("nan"), sigma=0.8)
CHANNEL_1024x256 = dict(nx=1024, ny=256, phi=0.5, Da=1e-2)


def batch_cases(n: int = 512, seed: int = 7, side_lo: int = 64, side_hi: int = 1024,
                max_aspect: float = 4.0, pr: float = 0.71):
    """Seeded batch of independent cavities: side lengths log-uniform in
    [side_lo, side_hi], aspect ratio uniform in [1, max_aspect] (the long side
    is drawn, the short one divided by the aspect, both at least 8),
    log10 Ra in [3, 6], log10 Da in [-4, -1], porosity in [0.4, 0.9],
    sigma in [0.5, 2].  Returns a list of CavityCase."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        side = int(round(math.exp(rng.uniform(math.log(side_lo), math.log(side_hi)))))
        aspect = rng.uniform(1.0, max_aspect)
        short = max(8, int(round(side / aspect)))
        if rng.uniform() < 0.5:
            nx, ny = side, short
        else:
            nx, ny = short, side
        out.append(CavityCase(nx=nx, ny=ny, Ra=10 ** rng.uniform(3, 6), Da=10 ** rng.uniform(-4, -1),
                              Pr=pr, phi=rng.uniform(0.4, 0.9), sigma=rng.uniform(0.5, 2.0)))
    return out


def warmstart_cases(n: int = 2200, seed: int = 11, size: int = 128, ell: float = 16.0, amp: float = 0.1,
                    pr_lo: float = 0.7, pr_hi: float = 1.0):
    """Seeded square cavities for the learned warm start: log10 Ra in [3, 6],
    log10 Da in [-4, -1], mean porosity in [0.4, 0.9], sigma in [0.5, 2],
    Pr uniform in [pr_lo, pr_hi]; each case has its own porosity field
    eps(x) = clip(mean + amp * g(x), 0.3, 0.95), g a unit Gaussian random
    field (correlation length ell) with seed seed * 100003 + case index.
    Returns a list of (CavityCase, (size, size) porosity field)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        ra, da = 10 ** rng.uniform(3, 6), 10 ** rng.uniform(-4, -1)
        mean, sg, pr = rng.uniform(0.4, 0.9), rng.uniform(0.5, 2.0), rng.uniform(pr_lo, pr_hi)
        g = gaussian_random_field(size, size, ell, seed * 100003 + i)
        phi = np.ascontiguousarray(np.clip(mean + amp * g, 0.3, 0.95))
        out.append((CavityCase(nx=size, ny=size, Ra=ra, Da=da, Pr=pr, phi=mean, sigma=sg), phi))
    return out
