"""ctypes front end of the FP64 C projectors in ``ctg_oracle.c``.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The discretisation (grid, Joseph A, pixel-driven B) is the one documented at
the top of ``ctg_oracle.c``; Sec. 1 eq. (1.1)-(1.2) of the paper fixes the
shapes A in R^{m x n}, B in R^{n x m}, m = N_a * N_d, n = N^2.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ctg_oracle.c")
_LIB = os.path.join(_HERE, "libctg_oracle.so")
_lib = None


def build_library(force: bool = False) -> str:
    """Compile ctg_oracle.c with gcc (-O2, OpenMP) next to this file."""
    if force or not os.path.exists(_LIB) or \
            os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                        "-D_DEFAULT_SOURCE", _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_library())
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        g = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
             ctypes.c_double, ctypes.c_double, ctypes.c_double]
        lib.orc_angles.argtypes = g + [dp, dp, i32p]
        lib.orc_angles.restype = ctypes.c_int
        lib.orc_forward.argtypes = g + [dp, dp]
        lib.orc_forward.restype = ctypes.c_int
        lib.orc_backproject.argtypes = g + [dp, dp]
        lib.orc_backproject.restype = ctypes.c_int
        lib.orc_forward_triplets.argtypes = g + [i64p, i64p, dp]
        lib.orc_forward_triplets.restype = ctypes.c_long
        lib.orc_backproject_triplets.argtypes = g + [i64p, i64p, dp]
        lib.orc_backproject_triplets.restype = ctypes.c_long
        _lib = lib
    return _lib


@dataclass(frozen=True)
class Geometry:
    """2D parallel-beam geometry; pixel size 1, integer start/range degrees."""
    N: int
    n_angles: int
    n_det: int
    angle_start_deg: float = 0.0
    angle_range_deg: float = 180.0
    det_spacing: float = 1.0

    @property
    def n(self) -> int:
        return self.N * self.N

    @property
    def m(self) -> int:
        return self.n_angles * self.n_det

    def _args(self):
        return (self.N, self.n_angles, self.n_det, float(self.angle_start_deg),
                float(self.angle_range_deg), float(self.det_spacing))


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _check(rc):
    if rc < 0:
        raise ValueError("invalid geometry (integer start/range degrees, "
                         "positive sizes and spacing are required)")
    return rc


def angles(g: Geometry):
    """(cos, sin, row_driven) per angle, FP64 / int32."""
    c = np.empty(g.n_angles)
    s = np.empty(g.n_angles)
    rd = np.empty(g.n_angles, dtype=np.int32)
    _check(_load().orc_angles(*g._args(), _ptr(c, ctypes.c_double),
                              _ptr(s, ctypes.c_double), _ptr(rd, ctypes.c_int32)))
    return c, s, rd


def forward(g: Geometry, x) -> np.ndarray:
    """b = A x (matrix-free FP64 Joseph projector); x of length n or (N, N)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1))
    assert x.size == g.n
    b = np.empty(g.m)
    _check(_load().orc_forward(*g._args(), _ptr(x, ctypes.c_double),
                               _ptr(b, ctypes.c_double)))
    return b


def backproject(g: Geometry, b) -> np.ndarray:
    """x = B b (matrix-free FP64 pixel-driven back projector)."""
    b = np.ascontiguousarray(np.asarray(b, dtype=np.float64).reshape(-1))
    assert b.size == g.m
    x = np.empty(g.n)
    _check(_load().orc_backproject(*g._args(), _ptr(b, ctypes.c_double),
                                   _ptr(x, ctypes.c_double)))
    return x


def _triplets(fn, g: Geometry, cap: int, shape):
    rows = np.empty(cap, dtype=np.int64)
    cols = np.empty(cap, dtype=np.int64)
    vals = np.empty(cap)
    nnz = _check(fn(*g._args(), _ptr(rows, ctypes.c_int64),
                    _ptr(cols, ctypes.c_int64), _ptr(vals, ctypes.c_double)))
    return sp.csr_matrix((vals[:nnz], (rows[:nnz], cols[:nnz])), shape=shape)


def matrix_A(g: Geometry) -> sp.csr_matrix:
    """Explicit sparse A (m x n), for small geometries."""
    return _triplets(_load().orc_forward_triplets, g, 2 * g.m * g.N, (g.m, g.n))


def matrix_B(g: Geometry) -> sp.csr_matrix:
    """Explicit sparse B (n x m), for small geometries."""
    return _triplets(_load().orc_backproject_triplets, g, 2 * g.n * g.n_angles,
                     (g.n, g.m))


def matrix_B_tau(g: Geometry, tau: float) -> sp.csr_matrix:
    """The thresholded back projector of Sec. 6.5, eq. (Btau):
    (B_tau)_ij = A_ji if A_ji >= tau * max_ij A_ij, else 0 (all entries of A
    are >= 0).  tau = 0 gives the matched back projector A^T."""
    A = matrix_A(g).tocoo()
    thr = tau * A.data.max()
    keep = A.data >= thr
    return sp.csr_matrix((A.data[keep], (A.col[keep], A.row[keep])), shape=(g.n, g.m))
