"""ctypes declarations of the C ABI in ``include/se_gb300.h``.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

SE_WIN_GAUSSIAN, SE_WIN_PKB = 0, 1
SE_F32, SE_F64 = 0, 1
SE_ADD_SELF, SE_CHECK_NEUTRAL, SE_SYNC_CHECK, SE_HOST_IO = 1, 2, 4, 8
SE_BATCH_NO_AUTOTUNE, SE_BATCH_BRANCHES, SE_BATCH_FUSED, SE_BATCH_LINES = 1, 2, 4, 8
SE_ACCUMULATE = 16

STATUS = {0: "SE_OK", 1: "SE_EINVAL", 2: "SE_ENONNEUTRAL", 3: "SE_EOUTOFBOX", 4: "SE_ENOMEM",
          5: "SE_ECUDA", 6: "SE_ECUFFT", 7: "SE_ETIMEOUT", 8: "SE_ENOTFINITE", 9: "SE_ECAPACITY"}

# every symbol declared in include/se_gb300.h
EXPORTS = ["se_opts_default", "se_plan_create", "se_plan_destroy", "se_plan_set_stream", "se_plan_reserve",
           "se_plan_get_info", "se_plan_check", "se_potential", "se_force", "se_vjp",
           "se_plan_set_profiling", "se_plan_get_profile", "se_potential_noalloc",
           "se_batch_create", "se_batch_destroy", "se_batch_set_stream", "se_batch_force", "se_batch_force_each",
           "se_batch_get_system", "se_batch_get_form", "se_batch_get_accuracy", "se_real_space",
           "se_params_from_tolerance", "se_measure_peak", "se_debug_fail_alloc", "se_status_str", "se_last_error"]
SE_N_STAGES = 8
STAGES = ["bin", "spread", "merge", "fft_fwd", "scale", "fft_inv", "gather", "energy"]


class SEError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.name = STATUS.get(code, str(code))


class Opts(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("s0", ctypes.c_double), ("s_mt", ctypes.c_int),
                ("n_l", ctypes.c_int), ("nu", ctypes.c_int), ("shape", ctypes.c_double),
                ("aft_eps", ctypes.c_double), ("tile", ctypes.c_int), ("spread_mode", ctypes.c_int),
                ("gather_mode", ctypes.c_int), ("split", ctypes.c_int),
                ("force_method", ctypes.c_int), ("fft_mode", ctypes.c_int), ("fft_sizes", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("D", ctypes.c_int), ("M", ctypes.c_int), ("P", ctypes.c_int), ("nu", ctypes.c_int),
                ("Mt", ctypes.c_int), ("s0_mt", ctypes.c_int), ("s_mt", ctypes.c_int), ("n_l", ctypes.c_int),
                ("grid", ctypes.c_int * 3), ("tile", ctypes.c_int * 3), ("n_tiles", ctypes.c_int),
                ("h", ctypes.c_double), ("L", ctypes.c_double), ("Lt", ctypes.c_double), ("R", ctypes.c_double),
                ("delta_L", ctypes.c_double), ("xi", ctypes.c_double), ("shape", ctypes.c_double),
                ("capacity", ctypes.c_int64), ("device_bytes", ctypes.c_int64), ("column_fft", ctypes.c_int),
                ("M_v", ctypes.c_int * 3), ("Mt_v", ctypes.c_int * 3), ("s0_mt_v", ctypes.c_int * 3),
                ("s_mt_v", ctypes.c_int * 3), ("n_I", ctypes.c_int * 3), ("L_v", ctypes.c_double * 3)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load the shared library; raise if it is missing (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library {path} is not built; run __graft_entry__.build() "
                               "or python -m paper_1712_04732_gb300.build")
        _build.build()
    lib = ctypes.CDLL(path)
    vp, i64, ci, cd, cu = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_uint
    sigs = {
        "se_opts_default": (None, [ctypes.POINTER(Opts)]),
        "se_plan_create": (ci, [ctypes.POINTER(vp), ctypes.POINTER(cd), ci, cd, ci, ci, ci, ci, ctypes.POINTER(Opts)]),
        "se_plan_destroy": (ci, [vp]),
        "se_plan_set_stream": (ci, [vp, vp]),
        "se_plan_reserve": (ci, [vp, i64]),
        "se_plan_get_info": (ci, [vp, ctypes.POINTER(Info)]),
        "se_plan_check": (ci, [vp]),
        "se_potential": (ci, [vp, i64, vp, vp, vp, cu]),
        "se_force": (ci, [vp, i64, vp, vp, vp, vp, vp, cu]),
        "se_vjp": (ci, [vp, i64, vp, vp, vp, vp, vp]),
        "se_plan_set_profiling": (ci, [vp, ci]),
        "se_potential_noalloc": (ci, [vp, i64, vp, vp, vp, cu]),
        "se_real_space": (ci, [vp, i64, vp, vp, cd, vp, vp, cu]),
        "se_batch_create": (ci, [ctypes.POINTER(vp), ci, vp, vp, vp, vp, vp, cd, ci, ci, cu]),
        "se_batch_destroy": (ci, [vp]),
        "se_batch_set_stream": (ci, [vp, vp]),
        "se_batch_force": (ci, [vp, vp, vp, vp, vp, vp]),
        "se_batch_force_each": (ci, [vp, vp, vp, vp, vp, vp]),
        "se_batch_get_system": (ci, [vp, ci, ctypes.POINTER(Info)]),
        "se_batch_get_form": (ci, [vp, ctypes.POINTER(ci), ctypes.POINTER(i64)]),
        "se_batch_get_accuracy": (ci, [vp, ci, ctypes.POINTER(cd), ctypes.POINTER(cd)]),
        "se_plan_get_profile": (ci, [vp, ctypes.POINTER(cd), ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "se_params_from_tolerance": (ci, [cd, cd, ctypes.c_int64, cd, ctypes.POINTER(cd), ci, ci,
                                          ctypes.POINTER(ci), ctypes.POINTER(ci)]),
        "se_measure_peak": (ci, [ci, i64, ctypes.POINTER(cd), ctypes.POINTER(cd)]),
        "se_debug_fail_alloc": (ci, [i64]),
        "se_status_str": (ctypes.c_char_p, [ci]),
        "se_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def check(code: int) -> None:
    if code != 0:
        msg = load().se_last_error().decode(errors="replace")
        raise SEError(code, msg)
