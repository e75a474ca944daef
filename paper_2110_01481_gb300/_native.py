"""ctypes binding of libctgmres (include/ctgmres.h): argument marshalling only.

Every computation runs in the CUDA library; this module only converts torch
CUDA tensors to device pointers and structs.  Importing it raises if the
compiled library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libctgmres.so")

CTG_OK = 0
CTG_ERR_INVALID_ARG = -1
CTG_ERR_OOM = -2
CTG_ERR_CUDA = -3
CTG_ERR_TIMEOUT = -4
CTG_ERR_WORKSPACE = -5
CTG_ERR_BUSY = -6
CTG_AB, CTG_BA, CTG_LSQR, CTG_LSMR = 0, 1, 2, 3
VARIANTS = {"ab": CTG_AB, "ba": CTG_BA, "lsqr": CTG_LSQR, "lsmr": CTG_LSMR}
CTG_STOP_MAXIT, CTG_STOP_DP, CTG_STOP_BREAKDOWN = 0, 1, 2
CTG_BASIS_FP32, CTG_BASIS_BF16, CTG_BASIS_FP16 = 0, 1, 2
BACK = {"pixel": 0, "matched": 1, "threshold": 2}
RULES = {"dp": 0, "ncp": 1}
CTG_STOP_NCP = 3
BASIS = {"fp32": CTG_BASIS_FP32, "bf16": CTG_BASIS_BF16, "fp16": CTG_BASIS_FP16}


class CtgGeom(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("n_angles", ctypes.c_int32),
                ("n_det", ctypes.c_int32), ("back_model", ctypes.c_int32),
                ("angle_start_deg", ctypes.c_double),
                ("angle_range_deg", ctypes.c_double),
                ("det_spacing", ctypes.c_double),
                ("back_tau", ctypes.c_double)]


class CtgTuning(ctypes.Structure):
    _fields_ = [("fwd_angles", ctypes.c_int32), ("back_chunk", ctypes.c_int32),
                ("tuned", ctypes.c_int32), ("fwd_us", ctypes.c_float * 2),
                ("back_us", ctypes.c_float * 3), ("fwd_warp_angles", ctypes.c_int32),
                ("fwd_split_us", ctypes.c_float * 2)]


class CtgOpts(ctypes.Structure):
    _fields_ = [("maxit", ctypes.c_int32), ("basis_dtype", ctypes.c_int32),
                ("tau", ctypes.c_double), ("noise_norm", ctypes.c_double),
                ("stop_rule", ctypes.c_int32)]


class CtgInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("stop_reason", ctypes.c_int32),
                ("resnorm", ctypes.c_double), ("rho", ctypes.c_double),
                ("history", ctypes.POINTER(ctypes.c_double)),
                ("ncp_history", ctypes.POINTER(ctypes.c_double))]


class CtgTiming(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 4), ("calls", ctypes.c_int64 * 4),
                ("kernels", ctypes.c_int64)]


PHASES = ("forward", "back", "arnoldi", "other")


class CtgLayout(ctypes.Structure):
    _fields_ = [("off_w", ctypes.c_size_t), ("ld_w", ctypes.c_size_t),
                ("off_h", ctypes.c_size_t), ("total_bytes", ctypes.c_size_t)]


EXPORTS = ("ctg_create", "ctg_destroy", "ctg_project", "ctg_backproject", "ctg_ncp_distance", "ctg_set_tiles", "ctg_set_fwd_tiles", "ctg_get_tuning",
           "ctg_workspace_bytes", "ctg_workspace_layout", "ctg_ab_gmres",
           "ctg_ba_gmres", "ctg_lsqr", "ctg_lsmr", "ctg_cgs2_scratch_bytes", "ctg_cgs2", "ctg_cgs2_noalloc",
           "ctg_set_timing", "ctg_get_timing", "ctg_set_wait_limit", "ctg_status_string",
           "ctg_batch_create", "ctg_batch_workspace_bytes", "ctg_batch_solve", "ctg_batch_destroy",
           "ctg_engine_create", "ctg_engine_request_bytes", "ctg_engine_submit",
           "ctg_engine_step", "ctg_engine_in_flight", "ctg_engine_destroy")


def _declare(lib):
    vp, sz, i32, i64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32, ctypes.c_int64
    G, O = ctypes.POINTER(CtgGeom), ctypes.POINTER(CtgOpts)
    lib.ctg_create.argtypes = [ctypes.POINTER(vp)]
    lib.ctg_create.restype = ctypes.c_int
    lib.ctg_destroy.argtypes = [vp]
    lib.ctg_destroy.restype = None
    for f in (lib.ctg_project, lib.ctg_backproject):
        f.argtypes = [vp, G, vp, vp, vp]
        f.restype = ctypes.c_int
    lib.ctg_workspace_bytes.argtypes = [G, ctypes.c_int, O]
    lib.ctg_workspace_bytes.restype = sz
    lib.ctg_workspace_layout.argtypes = [G, ctypes.c_int, O, ctypes.POINTER(CtgLayout)]
    lib.ctg_workspace_layout.restype = ctypes.c_int
    for f in (lib.ctg_ab_gmres, lib.ctg_ba_gmres, lib.ctg_lsqr, lib.ctg_lsmr):
        f.argtypes = [vp, G, vp, vp, vp, O, vp, sz, ctypes.POINTER(CtgInfo), vp]
        f.restype = ctypes.c_int
    lib.ctg_cgs2_scratch_bytes.argtypes = [i64, i32]
    lib.ctg_cgs2_scratch_bytes.restype = sz
    lib.ctg_cgs2.argtypes = [vp, i64, i64, i32, vp, vp, vp, vp, sz, vp]
    lib.ctg_cgs2.restype = ctypes.c_int
    lib.ctg_cgs2_noalloc.argtypes = [vp, i64, i64, i32, vp, vp, vp, vp]
    lib.ctg_cgs2_noalloc.restype = ctypes.c_int
    lib.ctg_set_timing.argtypes = [vp, ctypes.c_int]
    lib.ctg_set_timing.restype = ctypes.c_int
    lib.ctg_set_wait_limit.argtypes = [vp, i64]
    lib.ctg_set_wait_limit.restype = ctypes.c_int
    lib.ctg_get_timing.argtypes = [vp, ctypes.POINTER(CtgTiming), ctypes.c_int]
    lib.ctg_get_timing.restype = ctypes.c_int
    lib.ctg_batch_create.argtypes = [vp, i32, G, ctypes.POINTER(i32), O, ctypes.POINTER(vp)]
    lib.ctg_batch_create.restype = ctypes.c_int
    lib.ctg_batch_workspace_bytes.argtypes = [vp]
    lib.ctg_batch_workspace_bytes.restype = sz
    lib.ctg_batch_solve.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                    ctypes.POINTER(CtgInfo), vp]
    lib.ctg_batch_solve.restype = ctypes.c_int
    lib.ctg_batch_destroy.argtypes = [vp]
    lib.ctg_batch_destroy.restype = None
    lib.ctg_engine_create.argtypes = [vp, i32, sz, ctypes.POINTER(vp)]
    lib.ctg_engine_create.restype = ctypes.c_int
    lib.ctg_engine_request_bytes.argtypes = [G, i32, O]
    lib.ctg_engine_request_bytes.restype = sz
    lib.ctg_engine_submit.argtypes = [vp, G, i32, O, vp, vp, vp, ctypes.POINTER(ctypes.c_double),
                                      ctypes.c_int64, vp]
    lib.ctg_engine_submit.restype = ctypes.c_int
    lib.ctg_engine_step.argtypes = [vp, i32, i32, ctypes.POINTER(ctypes.c_int64),
                                    ctypes.POINTER(CtgInfo), ctypes.POINTER(i32)]
    lib.ctg_engine_step.restype = ctypes.c_int
    lib.ctg_engine_in_flight.argtypes = [vp]
    lib.ctg_engine_in_flight.restype = i32
    lib.ctg_engine_destroy.argtypes = [vp]
    lib.ctg_engine_destroy.restype = None
    lib.ctg_set_tiles.argtypes = [vp, i32, i32]
    lib.ctg_set_tiles.restype = ctypes.c_int
    lib.ctg_set_fwd_tiles.argtypes = [vp, i32, i32]
    lib.ctg_set_fwd_tiles.restype = ctypes.c_int
    lib.ctg_get_tuning.argtypes = [vp, G, ctypes.POINTER(CtgTuning)]
    lib.ctg_get_tuning.restype = ctypes.c_int
    lib.ctg_ncp_distance.argtypes = [vp, G, vp, ctypes.POINTER(ctypes.c_double), vp]
    lib.ctg_ncp_distance.restype = ctypes.c_int
    lib.ctg_status_string.argtypes = [ctypes.c_int]
    lib.ctg_status_string.restype = ctypes.c_char_p
    return lib


_lib = None


def lib():
    """The loaded library; raises ImportError if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` "
                "(this package has no CPU fallback)")
        _lib = _declare(ctypes.CDLL(LIB_PATH))
    return _lib


class CtgError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {lib().ctg_status_string(status).decode()} ({status})")


def check(status: int, what: str) -> None:
    if status != CTG_OK:
        raise CtgError(status, what)
