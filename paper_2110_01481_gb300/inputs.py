"""Seeded synthetic inputs shared by the CUDA path and the FP64 oracle.

This module holds only input generation: phantoms (the ground truth x̄ of
eq. (1.1)) and the Gaussian noise e added to the noise-free data b̄ = A x̄.
It contains none of the method's arithmetic (no projector, no Krylov step),
imports nothing else from this package, and draws every random number from
numpy's PCG64 generator seeded by the caller.

Conventions (both sides use them):
  * image x has shape (N, N), row-major, x[i, j] with i = row, j = column;
    pixel (i, j) has centre (j - (N-1)/2, i - (N-1)/2) in pixel units;
  * phantom ellipse coordinates are normalised to [-1, 1]^2 and scaled by N/2;
  * sinogram b has shape (N_angles, N_det), angle-major.

The paper's own ground truth (AIR Tools' ``threephases`` phantom, Sec. 6.1)
is not available; the modified Shepp-Logan head phantom and seeded random
ellipses stand in for it, with values in [0, 1] like the paper's.
"""
from __future__ import annotations

import math

import numpy as np

# Modified Shepp-Logan head phantom (Shepp & Logan 1974 geometry with the
# higher-contrast intensity table of Toft 1996): ten additive ellipses,
# columns = intensity, semi-axis a, semi-axis b, centre x0, centre y0,
# rotation in degrees.  Values of the summed image lie in [0, 1].
_MODIFIED_SHEPP_LOGAN = (
    (1.00, 0.6900, 0.9200, 0.00, 0.0000, 0.0),
    (-0.80, 0.6624, 0.8740, 0.00, -0.0184, 0.0),
    (-0.20, 0.1100, 0.3100, 0.22, 0.0000, -18.0),
    (-0.20, 0.1600, 0.4100, -0.22, 0.0000, 18.0),
    (0.10, 0.2100, 0.2500, 0.00, 0.3500, 0.0),
    (0.10, 0.0460, 0.0460, 0.00, 0.1000, 0.0),
    (0.10, 0.0460, 0.0460, 0.00, -0.1000, 0.0),
    (0.10, 0.0460, 0.0230, -0.08, -0.6050, 0.0),
    (0.10, 0.0230, 0.0230, 0.00, -0.6060, 0.0),
    (0.10, 0.0230, 0.0460, 0.06, -0.6050, 0.0),
)


def _pixel_grid(N: int):
    """Normalised pixel-centre coordinates (X, Y) in [-1, 1], shape (N, N)."""
    c = (np.arange(N, dtype=np.float64) - (N - 1) / 2.0) / (N / 2.0)
    Y, X = np.meshgrid(c, c, indexing="ij")
    return X, Y


def _inside(X, Y, a, b, x0, y0, phi_rad):
    ct, st = math.cos(phi_rad), math.sin(phi_rad)
    xr = (X - x0) * ct + (Y - y0) * st
    yr = -(X - x0) * st + (Y - y0) * ct
    return (xr / a) ** 2 + (yr / b) ** 2 <= 1.0


def shepp_logan(N: int) -> np.ndarray:
    """Modified Shepp-Logan phantom sampled at pixel centres, float64 (N, N)."""
    X, Y = _pixel_grid(N)
    img = np.zeros((N, N), dtype=np.float64)
    for rho, a, b, x0, y0, phi in _MODIFIED_SHEPP_LOGAN:
        img[_inside(X, Y, a, b, x0, y0, math.radians(phi))] += rho
    # the additive table is exact in real arithmetic; clip the 1e-16 residue
    return np.clip(img, 0.0, 1.0)


def random_ellipse_params(seed: int, n_ellipses: int = 20) -> np.ndarray:
    """Seeded ellipse table, rows = (intensity, a, b, x0, y0, phi_rad).

    Centres uniform in the disc of radius 0.7, semi-axes uniform in
    [0.05, 0.4], rotation uniform in [0, pi), intensity uniform in [0, 1].
    """
    rng = np.random.default_rng(seed)
    r = 0.7 * np.sqrt(rng.uniform(0.0, 1.0, n_ellipses))
    t = rng.uniform(0.0, 2.0 * math.pi, n_ellipses)
    x0, y0 = r * np.cos(t), r * np.sin(t)
    a = rng.uniform(0.05, 0.4, n_ellipses)
    b = rng.uniform(0.05, 0.4, n_ellipses)
    phi = rng.uniform(0.0, math.pi, n_ellipses)
    rho = rng.uniform(0.0, 1.0, n_ellipses)
    return np.stack([rho, a, b, x0, y0, phi], axis=1)


def random_ellipses(N: int, seed: int, n_ellipses: int = 20) -> np.ndarray:
    """Painter's-order random-ellipse phantom (later ellipses overwrite),
    background 0, values in [0, 1]; float64 (N, N)."""
    X, Y = _pixel_grid(N)
    img = np.zeros((N, N), dtype=np.float64)
    for rho, a, b, x0, y0, phi in random_ellipse_params(seed, n_ellipses):
        img[_inside(X, Y, a, b, x0, y0, phi)] = rho
    return img


def single_ellipse(N: int, rho: float, a: float, b: float, x0: float,
                   y0: float, phi_rad: float) -> np.ndarray:
    """One ellipse (normalised units) sampled at pixel centres."""
    X, Y = _pixel_grid(N)
    img = np.zeros((N, N), dtype=np.float64)
    img[_inside(X, Y, a, b, x0, y0, phi_rad)] = rho
    return img


def noise_direction(m: int, seed: int) -> np.ndarray:
    """Unit-norm white Gaussian direction g/||g||, g ~ N(0, I_m), PCG64(seed)."""
    g = np.random.default_rng(seed).standard_normal(m)
    return g / np.linalg.norm(g)


def add_noise(b_bar: np.ndarray, eta: float, seed: int):
    """b = b̄ + e with ||e|| / ||b̄|| = eta exactly (white Gaussian, Sec. 6.1).

    Returns (b, ||e||)."""
    b_bar = np.asarray(b_bar, dtype=np.float64)
    e = eta * np.linalg.norm(b_bar) * noise_direction(b_bar.size, seed)
    e = e.reshape(b_bar.shape)
    return b_bar + e, float(np.linalg.norm(e))


def detector_count(N: int) -> int:
    """N_det = ceil(sqrt(2) * N), the detector width that covers the image."""
    return int(math.ceil(math.sqrt(2.0) * N))
