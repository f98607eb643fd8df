"""ctypes binding of ``libdmrg_rotate.so`` (declared in ``include/dmrg_rotate.h``).

Argument marshalling only: every step of the rotation runs in the library's
CUDA kernels.  Loading fails loudly when the library has not been built; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdmrg_rotate.so")

DMRG_OK = 0
STATUS = {0: "DMRG_OK", 1: "DMRG_ERR_INVALID_ARG", 2: "DMRG_ERR_SHAPE",
          3: "DMRG_ERR_NOT_ORTHONORMAL", 4: "DMRG_ERR_WORKSPACE", 5: "DMRG_ERR_CUDA",
          6: "DMRG_ERR_TIMEOUT", 7: "DMRG_ERR_UNSUPPORTED"}
PRECISION = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16x3": 3}
OPTION = {"graph": 1, "kernel_timing": 2, "wait_timeout_ms": 3, "check_ortho": 4,
          "test_withhold_arrival": 5, "deterministic": 6, "accum_chain": 7, "blocked_small": 8,
          "truncation_jacobi": 9, "fused_rotation": 10, "pack_operators": 11,
          "store_epilogue": 12}

_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_int = ctypes.c_int
_sz = ctypes.c_size_t
_dbl = ctypes.c_double


class DmrgQnSector(ctypes.Structure):
    _fields_ = [("n_up", ctypes.c_int32), ("n_dn", ctypes.c_int32), ("dim", ctypes.c_int64)]


class DmrgQnShift(ctypes.Structure):
    _fields_ = [("d_up", ctypes.c_int32), ("d_dn", ctypes.c_int32)]


# name -> (argtypes); every entry point returns dmrg_status (int) unless listed below
SIGNATURES = {
    "dmrg_create": [ctypes.POINTER(_p)],
    "dmrg_destroy": [_p],
    "dmrg_sync_status": [_p, _p],
    "dmrg_set_option": [_p, _int, _dbl],
    "dmrg_kernel_timing": [_p, ctypes.c_char_p, _sz, _int],
    "dmrg_rotate_ops_workspace": [_p, _i64, _i64, _int, _i64, _int, ctypes.POINTER(_sz)],
    "dmrg_rotate_ops": [_p, _p, _i64, _int, _i64, _p, _int, _i64, _p, _int, _p, _sz, _p],
    "dmrg_autotune_rotate_ops": [_p, _p, _i64, _int, _i64, _p, _int, _i64, _p, _int, _p, _sz, _p],
    "dmrg_rotate_ops_backward_workspace": [_p, _i64, _i64, _int, _i64, _int, ctypes.POINTER(_sz)],
    "dmrg_rotate_ops_backward": [_p, _p, _i64, _int, _i64, _p, _p, _int, _i64, _p, _p, _int, _p,
                                 _sz, _p],
    "dmrg_orthonormality_error": [_p, _p, _i64, _i64, _p, _p, _sz, _p],
    "dmrg_orthonormality_error_workspace": [_p, _i64, _i64, ctypes.POINTER(_sz)],
    "dmrg_correlations_workspace": [_p, _i64, _i64, ctypes.POINTER(_sz)],
    "dmrg_correlations": [_p, _p, _int, _p, _i64, _i64, _p, _p, _sz, _p],
    "dmrg_blocked_plan_create": [_p, ctypes.POINTER(DmrgQnSector), _i32, ctypes.POINTER(DmrgQnShift),
                                 _i32, ctypes.POINTER(DmrgQnSector), _i32,
                                 ctypes.POINTER(DmrgQnShift), _i64, ctypes.POINTER(_p)],
    "dmrg_blocked_plan_destroy": [_p],
    "dmrg_blocked_plan_sizes": [_p, _int, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                ctypes.POINTER(_i64), ctypes.POINTER(_sz)],
    "dmrg_blocked_plan_stats": [_p, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                ctypes.POINTER(_dbl)],
    "dmrg_rotate_ops_blocked": [_p, _p, _p, _p, _int, _p, _int, _p, _sz, _p],
    "dmrg_rotate_ops_noalloc": [_p, _i64, _int, _i64, _p, _int, _i64, _p, _int, _p],
    "dmrg_debug_reciprocal": [_p, _p, _i64, _p],
    "dmrg_rotate_ops_host_workspace": [_p, _i64, _i64, _int, _i64, _int, _int, _i64,
                                       ctypes.POINTER(_sz)],
    "dmrg_rotate_ops_host": [_p, _p, _i64, _int, _i64, _p, _int, _i64, _p, _int, _i64, _p, _sz, _p],
    "dmrg_expectation_workspace": [_p, _i64, _i64, _i64, _int, ctypes.POINTER(_sz)],
    "dmrg_expectation": [_p, _p, _int, _i64, _p, _i64, _i64, _int, _p, _p, _sz, _p],
    "dmrg_cross_correlations_workspace": [_p, _i64, _i64, _i64, _i64, _int, _int, ctypes.POINTER(_sz)],
    "dmrg_cross_correlations": [_p, _p, _int, _i64, _p, _int, _i64, _p, _i64, _i64, _p, _p, _sz, _p],
    "dmrg_structure_factor": [_p, _p, _p, ctypes.c_double, _i64, _p, _p, _p],
    "dmrg_truncation_workspace": [_p, _i64, _i64, ctypes.POINTER(_sz)],
    "dmrg_truncation": [_p, _p, _i64, _i64, _i64, _p, _p, _p, ctypes.c_double, _int,
                        ctypes.POINTER(_int), _p, _sz, _p],
    "dmrg_rotate_site_ops_workspace": [_p, _i64, _i64, _int, _i64, _int, ctypes.POINTER(_sz)],
    "dmrg_rotate_site_ops": [_p, _p, _i64, _int, _i64, _p, _int, _i64, _int, _p, _p, _p, _p, _p, _int,
                             _p, _sz, _p],
}
STRING_RETURN = {"dmrg_status_string": [_int], "dmrg_last_error": [_p]}

_lock = threading.Lock()
_lib = None


def load():
    """Loads the library (built by ``paper_0909_5662_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                "libdmrg_rotate.so is not built (%s); run __graft_entry__.build() or "
                "python -m paper_0909_5662_gb300.build" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, argt in SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = argt
            f.restype = _int
        for name, argt in STRING_RETURN.items():
            f = getattr(lib, name)
            f.argtypes = argt
            f.restype = ctypes.c_char_p
        _lib = lib
        return lib


def exported_names():
    return list(SIGNATURES) + list(STRING_RETURN)


class DmrgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


def check(status: int, handle=None, what: str = ""):
    if status != DMRG_OK:
        lib = load()
        detail = lib.dmrg_last_error(handle).decode() if handle else ""
        raise DmrgError(status, (what + ": " if what else "") + detail)
