"""ctypes loader for ``librtcc3.so`` (argument marshalling only).

The library is the product: every step of the RT-CC3 path runs in its CUDA
kernels.  Loading fails loudly when the shared library is missing; there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "lib", "librtcc3.so")

OK = 0
ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NONFINITE, ERR_TIMEOUT, ERR_NOT_CONVERGED, ERR_STATE = (
    -1, -2, -3, -4, -5, -6, -7)
PREC_FP64, PREC_FP32, PREC_TF32, PREC_BF16 = 0, 1, 2, 3
FIELD_NONE, FIELD_STATIC, FIELD_COS, FIELD_GAUSS, FIELD_LRCW, FIELD_QRCW = 0, 1, 2, 3, 4, 5

_STATUS_NAMES = {ERR_ARG: "RTCC3_ERR_ARG", ERR_OOM: "RTCC3_ERR_OOM", ERR_CUDA: "RTCC3_ERR_CUDA",
                 ERR_NONFINITE: "RTCC3_ERR_NONFINITE", ERR_TIMEOUT: "RTCC3_ERR_TIMEOUT",
                 ERR_NOT_CONVERGED: "RTCC3_ERR_NOT_CONVERGED", ERR_STATE: "RTCC3_ERR_STATE"}


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("triples", ctypes.c_int), ("device", ctypes.c_int),
                ("use_graphs", ctypes.c_int), ("field_tol", ctypes.c_double),
                ("field_solver", ctypes.c_int), ("triples_chunk", ctypes.c_int),
                ("spin_budget", ctypes.c_longlong), ("eig_sweep_cap", ctypes.c_int),
                ("tc_scope", ctypes.c_int), ("storage", ctypes.c_int), ("checked", ctypes.c_int),
                ("serial", ctypes.c_int)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_longlong), ("ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


#: Every exported symbol with (restype, argtypes); mirrors include/rtcc3.h.
_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_DP = ctypes.POINTER(ctypes.c_double)
_LLP = ctypes.POINTER(ctypes.c_longlong)
SIGNATURES = {
    "rtcc3_default_options": (None, [ctypes.POINTER(Options)]),
    "rtcc3_create": (_I, [_I, _I, _I, ctypes.POINTER(Options), ctypes.POINTER(_P)]),
    "rtcc3_destroy": (_I, [_P]),
    "rtcc3_last_error": (ctypes.c_char_p, [_P]),
    "rtcc3_set_hamiltonian": (_I, [_P, _DP, _I, _DP, _DP]),
    "rtcc3_set_hamiltonian_eri": (_I, [_P, _DP, _DP, _DP]),
    "rtcc3_eri_cholesky": (_I, [_I, _DP, _D, _I, _DP, ctypes.POINTER(ctypes.c_int)]),
    "rtcc3_set_field": (_I, [_P, _I, _I, _D, _D, _D, _D, _DP]),
    "rtcc3_set_amplitudes": (_I, [_P, _I, _DP, _DP, _DP, _DP]),
    "rtcc3_get_amplitudes": (_I, [_P, _I, _DP, _DP, _DP, _DP]),
    "rtcc3_set_time": (_I, [_P, _D]),
    "rtcc3_get_time": (_I, [_P, _DP]),
    "rtcc3_compute_residuals": (_I, [_P, _I, _D, _DP, _DP, _DP, _DP, _DP, _DP]),
    "rtcc3_solve_ground_state": (_I, [_P, _D, _I]),
    "rtcc3_propagate_rk4": (_I, [_P, _D, _I, _DP, _DP]),
    "rtcc3_propagate_rk4_dev": (_I, [_P, _D, _I, _P, _P, _P]),
    "rtcc3_propagate_rk4_chunk": (_I, [_P, _D, _I, _DP, _DP]),
    "rtcc3_propagate_rk4_chunk_dev": (_I, [_P, _D, _I, _P, _P, _P]),
    "rtcc3_triples_forward_dev": (_I, [_P, _I, _D, _P, _P, _P, _P, _P]),
    "rtcc3_triples_vjp_dev": (_I, [_P, _I, _D, _P, _P, _P, _P, _P, _P, _P]),
    "rtcc3_triples_forward_noalloc_dev": (_I, [_P, _I, _D, _P, _P, _P, _P, _P]),
    "rtcc3_state_size": (_I, [_P, _LLP]),
    "rtcc3_get_state": (_I, [_P, _P, ctypes.c_longlong]),
    "rtcc3_set_state": (_I, [_P, _P, ctypes.c_longlong]),
    "rtcc3_stats": (_I, [_P, _LLP, _LLP]),
    "rtcc3_set_wait_budgets": (_I, [_P, ctypes.c_longlong, _I]),
    "rtcc3_measure_peaks": (_I, [_I, _DP]),
    "rtcc3_ground_state_history": (_I, [_P, _DP, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "rtcc3_set_observables": (_I, [_P, _I, _DP]),
    "rtcc3_get_observables": (_I, [_P, _DP, ctypes.c_longlong]),
    "rtcc3_autotune_triples": (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_float), _I,
                                    ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_float),
                                    ctypes.POINTER(_I)]),
    "rtcc3_set_profiling": (_I, [_P, _I]),
    "rtcc3_kernel_stats": (_I, [_P, ctypes.POINTER(KernelStat), _I, ctypes.POINTER(_I)]),
}

_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load librtcc3 (building it first if the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        from . import build as _build
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class RTCC3Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code
