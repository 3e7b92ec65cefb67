"""Seeded log-normal permeability fields (stand-ins for the paper's benchmark
permeability, which is only shown as a figure, Section 6).

A zero-mean, unit-variance Gaussian field g with squared-exponential
covariance C(r) = exp(-((rx/lx)^2 + (ry/ly)^2) / 2) is drawn by circulant
embedding on a 2x-padded periodic grid (FFT of the covariance gives the
eigenvalues, negative round-off eigenvalues are clipped), cropped to the
physical grid and re-standardised. Permeability is kappa = exp(sigma * g), or,
when a contrast is requested, ln(kappa) is mapped affinely so that
max(kappa)/min(kappa) equals the contrast and the geometric midpoint is 1.
"""
from __future__ import annotations

import numpy as np


def _gaussian_field(nx: int, ny: int, hx: float, hy: float, lx: float, ly: float,
                    rng: np.random.Generator) -> np.ndarray:
    px, py = 2 * nx, 2 * ny
    ix = np.arange(px)
    iy = np.arange(py)
    dx = np.minimum(ix, px - ix) * hx
    dy = np.minimum(iy, py - iy) * hy
    cov = np.exp(-0.5 * ((dy[:, None] / ly) ** 2 + (dx[None, :] / lx) ** 2))
    eig = np.fft.fft2(cov).real
    eig = np.clip(eig, 0.0, None)
    white = rng.standard_normal((py, px)) + 1j * rng.standard_normal((py, px))
    g = np.fft.ifft2(np.sqrt(eig) * np.fft.fft2(white)).real
    g = g[:ny, :nx]
    g = (g - g.mean()) / g.std()
    return g


def lognormal_field(nx: int, ny: int, Lx: float, Ly: float, sigma: float,
                    corr: tuple[float, float], seed: int,
                    contrast: float | None = None) -> np.ndarray:
    """Per-cell permeability, lexicographic (x fastest), shape (nx*ny,)."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    g = _gaussian_field(nx, ny, Lx / nx, Ly / ny, corr[0], corr[1], rng)
    if contrast is None:
        lk = sigma * g
    else:
        lo, hi = g.min(), g.max()
        lk = ((g - lo) / (hi - lo) - 0.5) * np.log(contrast)
    return np.exp(lk).reshape(-1).astype(np.float64)


def layered_lognormal_field(nx: int, ny: int, nz: int, Lx: float, Ly: float,
                            sigma_range: tuple[float, float],
                            corr: tuple[float, float], seed: int) -> np.ndarray:
    """3D layered field: nz independent x-y layers, layer k with its own sigma
    drawn uniformly in sigma_range. Shape (nx*ny*nz,), x fastest, z slowest."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    out = np.empty((nz, ny, nx))
    for k in range(nz):
        sig = rng.uniform(*sigma_range)
        out[k] = np.exp(sig * _gaussian_field(nx, ny, Lx / nx, Ly / ny, corr[0], corr[1], rng))
    return out.reshape(-1)
