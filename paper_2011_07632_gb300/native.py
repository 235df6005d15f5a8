"""ctypes loader for libspdhss.so (the C ABI of include/spdhss.h).

Argument marshalling only: every call goes straight to the CUDA library.  Loading fails
loudly when the library has not been built; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspdhss.so")

OK, EINVAL, ENOMEM, NOT_SPD, NO_CONVERGENCE, NUMERIC, TIMEOUT, ECUDA = range(8)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "NOT_SPD", 4: "NO_CONVERGENCE",
                5: "NUMERIC", 6: "TIMEOUT", 7: "ECUDA"}
KERNELS = {"exp": 0, "gauss": 1, "matern32": 2, "imq": 3, "rpy": 4}
DOFS = {"rpy": 3}   # unknowns per point of a vector-valued kernel


class SpdhssError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class KernelDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("ell", ctypes.c_double), ("shift", ctypes.c_double)]


_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_D = ctypes.c_double
_PI64 = ctypes.POINTER(ctypes.c_int64)

# void (*)(void* user, int instance, spdhss_status status): pcg_solve_batched_ex's callback
DONE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int, ctypes.c_int)

_SIGS = {
    "h2_build": [_P, _I64, _I, KernelDesc, _I, _D, _P, ctypes.POINTER(_P)],
    "h2_matmul": [_P, _P, _P, _I, _I64, _P],
    "spdhss_kernel_eval": [KernelDesc, _P, _P, _I64, _P],
    "h2_info": [_P, _PI64],
    "h2_export_tree": [_P] + [_PI64] * 11,
    "h2_export_skeletons": [_P, _PI64, _PI64],
    "h2_destroy": [_P],
    "spdhss_build": [_P, _I, _I, _P, ctypes.c_uint64, _P, ctypes.POINTER(_P)],
    "spdhss_build_tol": [_P, _I, _D, _I, _P, ctypes.c_uint64, _P, ctypes.POINTER(_P)],
    "spdhss_build_precision": [_P, _I, _D, _I, _P, ctypes.c_uint64, _I, _P,
                               ctypes.POINTER(_P)],
    "hss_matmul": [_P, _P, _P, _I, _I64, _P],
    "hss_info": [_P, _PI64],
    "hss_destroy": [_P],
    "ulv_factor": [_P, _P, ctypes.POINTER(_P)],
    "ulv_solve": [_P, _P, _P, _I, _I64, _P],
    "ulv_destroy": [_P],
    "ulv_solve_noalloc": [_P, _P, _P, _I, _I64, _P],
    "h2_matmul_mixed": [_P, _P, _P, _I, _I64, _P],
    "pcg_solve_mixed": [_P, _P, _P, _P, _I, _I64, _D, _I, ctypes.POINTER(_I),
                        ctypes.POINTER(_D), _P],
    "pcg_solve": [_P, _P, _P, _P, _I, _I64, _D, _I, ctypes.POINTER(_I),
                  ctypes.POINTER(_D), _P],
    "spdhss_build_batched": [_I, ctypes.POINTER(_P), _PI64, ctypes.POINTER(_I),
                             ctypes.POINTER(KernelDesc), ctypes.POINTER(_I), ctypes.POINTER(_D),
                             ctypes.POINTER(_I), ctypes.POINTER(_I),
                             ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(_P),
                             ctypes.POINTER(_I), _P,
                             ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                             ctypes.POINTER(_I)],
    "spdhss_gemm_f32": [_I, _I, _I, _P, _I64, _I, _P, _I64, _I, _P, _I64, ctypes.c_float,
                        ctypes.c_float, _I, _P],
    "pcg_solve_batched": [_I, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                          ctypes.POINTER(_P), ctypes.POINTER(_I), _PI64, _D, _I,
                          ctypes.POINTER(_P), ctypes.POINTER(_P), _P, ctypes.POINTER(_I)],
    "pcg_solve_batched_mixed": [_I, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                                ctypes.POINTER(_P), ctypes.POINTER(_I), _PI64, _D, _I,
                                ctypes.POINTER(_P), ctypes.POINTER(_P), _P, ctypes.POINTER(_I)],
    "pcg_solve_batched_ex": [_I, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                             ctypes.POINTER(_P), ctypes.POINTER(_I), _PI64, _D, _I,
                             ctypes.POINTER(_P), ctypes.POINTER(_P), _P, ctypes.POINTER(_I), _I,
                             DONE_FN, _P],
}


def lib():
    """The loaded library; raises if it is missing (build it with build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libspdhss.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name, None)
            if f is None:
                continue
            f.argtypes = args
            f.restype = ctypes.c_int
        L.spdhss_last_error.restype = ctypes.c_char_p
        L.spdhss_last_error.argtypes = []
        L.spdhss_launch_count.restype = ctypes.c_int64
        L.spdhss_launch_count.argtypes = []
        L.spdhss_version.restype = ctypes.c_char_p
        L.spdhss_version.argtypes = []
        L.spdhss_profile.restype = None
        L.spdhss_profile.argtypes = [ctypes.c_int]
        L.spdhss_batched_stats.restype = None
        L.spdhss_batched_stats.argtypes = [_PI64]
        L.spdhss_profile_report.restype = ctypes.c_int64
        L.spdhss_profile_report.argtypes = [ctypes.c_char_p, ctypes.c_int64]
        L.spdhss_tuning_report.restype = ctypes.c_int64
        L.spdhss_tuning_report.argtypes = [ctypes.c_char_p, ctypes.c_int64]
        _lib = L
    return _lib


def check(status: int) -> None:
    if status != OK:
        raise SpdhssError(status, lib().spdhss_last_error().decode())


def launch_count() -> int:
    return int(lib().spdhss_launch_count())


def profile_report() -> dict:
    import json
    need = int(lib().spdhss_profile_report(None, 0))
    buf = ctypes.create_string_buffer(need + 16)
    lib().spdhss_profile_report(buf, need + 16)
    return json.loads(buf.value.decode())


def tuning_report() -> dict:
    """The autotuned launch variants of this process: {key: chosen variant}."""
    need = int(lib().spdhss_tuning_report(None, 0))
    buf = ctypes.create_string_buffer(need + 16)
    lib().spdhss_tuning_report(buf, need + 16)
    out = {}
    for line in buf.value.decode().splitlines():
        if " -> " in line:
            k, v = line.split(" -> ", 1)
            out[k] = int(v.split()[0])
    return out


def exported_symbols() -> list:
    return list(_SIGS) + ["spdhss_last_error", "spdhss_launch_count", "spdhss_version",
                          "spdhss_profile", "spdhss_profile_report", "spdhss_tuning_report",
                          "spdhss_batched_stats"]
