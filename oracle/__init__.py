"""FP64 CPU oracle for AB-GMRES / BA-GMRES with an unmatched back projector.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
reference that the CUDA library is checked against.  Only the tests, the
smoke check and the benchmark's CPU-baseline / reference leg may import it.
It shares no code, header, table or helper with the CUDA library and imports
nothing from it.

  projectors  matrix-free FP64 Joseph forward projector A and pixel-driven
              back projector B (C, OpenMP), their explicit sparse forms, and
              the thresholded back projectors B_tau of Sec. 6.5
  krylov      AB-GMRES and BA-GMRES exactly as the algorithm box of Sec. 2
              (MGS Arnoldi; CGS2 as an option), the discrepancy principle of
              Sec. 6.4, and LSQR / LSMR for the matched case of Sec. 5
  stopping    the NCP criterion of Sec. 6.4 (a reading of its citation)
"""
from .projectors import (Geometry, angles, forward, backproject, matrix_A,
                         matrix_B, matrix_B_tau, build_library)
from .krylov import ab_gmres, ba_gmres, lsqr, lsmr
from .stopping import ncp, ncp_distance, first_local_minimum

__all__ = ["Geometry", "angles", "forward", "backproject", "matrix_A",
           "matrix_B", "matrix_B_tau", "build_library", "ab_gmres", "ba_gmres", "lsqr", "lsmr",
           "ncp", "ncp_distance", "first_local_minimum"]
