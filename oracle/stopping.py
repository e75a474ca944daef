"""The NCP stopping criterion of Sec. 6.4 (plain numpy, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper defines the criterion only by citation: the residual b - A x_k is
judged by its normalised cumulative periodogram (NCP), and the iterations
stop when the residual looks most like white noise.  Reading taken here:

  * the residual is arranged as the sinogram, N_a projections of N_d bins,
    and each projection is one signal (the noise is white along the
    detector);
  * for a projection r (length N_d), with q = floor(N_d / 2), the
    periodogram is p_i = |rhat_i|^2, i = 1..q, rhat the DFT of r (the zero
    frequency is left out), and the NCP is c_i = (p_1 + ... + p_i) /
    (p_1 + ... + p_q);
  * white noise has the expected NCP c_i = i / q; the distance of a
    projection is ||c - (1..q)/q||_2 (0 for a projection with no residual
    outside the zero frequency), and the distance of the residual is the
    mean over the projections;
  * k_NCP is the first k >= 0 at which the distance stops decreasing, i.e.
    the smallest k with d_{k+1} > d_k (maxit when there is none).
"""
from __future__ import annotations

import numpy as np


def ncp(r: np.ndarray) -> np.ndarray:
    """NCP of one projection: c_1..c_q (q = len(r) // 2)."""
    r = np.asarray(r, dtype=np.float64)
    q = r.size // 2
    p = np.abs(np.fft.fft(r))[1:q + 1] ** 2
    s = p.sum()
    if s == 0.0:
        return np.arange(1, q + 1) / q
    return np.cumsum(p) / s


def ncp_distance(r: np.ndarray, n_angles: int, n_det: int) -> float:
    """Mean over the projections of ||c - (1..q)/q||_2."""
    R = np.asarray(r, dtype=np.float64).reshape(n_angles, n_det)
    q = n_det // 2
    line = np.arange(1, q + 1) / q
    return float(np.mean([np.linalg.norm(ncp(row) - line) for row in R]))


def first_local_minimum(d) -> int:
    """Smallest k with d[k+1] > d[k]; len(d) - 1 if d never increases."""
    for k in range(len(d) - 1):
        if d[k + 1] > d[k]:
            return k
    return len(d) - 1
