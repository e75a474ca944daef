"""GB300-native AB-GMRES / BA-GMRES for CT with an unmatched back projector.

Python front end of the CUDA library libctgmres (include/ctgmres.h).  Torch
is used for device memory and streams only; every step of the projectors and
of the Krylov solvers runs in the library's kernels.  See ``api`` for the
calls: ``project``, ``backproject``, ``ab_gmres``, ``ba_gmres``, ``cgs2``.
"""
__all__ = ["Geometry", "Context", "SolveResult", "Batch", "Engine", "project", "backproject", "ncp_distance",
           "ab_gmres", "ba_gmres", "lsqr", "lsmr", "cgs2", "workspace_bytes", "workspace_layout"]


def __getattr__(name):
    # the CUDA-backed API is imported lazily so that ``inputs`` (seeded data
    # generators) can be used without loading the library
    if name in __all__:
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
