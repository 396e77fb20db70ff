"""ctypes declarations of the C-ABI in include/sfcdd.h (argument marshalling only).

Loading fails loudly when libsfcdd.so has not been built: there is no CPU or
eager fallback for any step of the solver.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsfcdd.so")

SFCDD_OK = 0
STATUS = {
    0: "OK", -1: "INVALID_ARG", -2: "KEY_OVERFLOW", -3: "NOMEM", -4: "NOT_SPD", -5: "MAXIT",
    -6: "NAN", -7: "TIMEOUT", -8: "CUDA", -9: "UNSUPPORTED",
}
PRECISION = {"fp64": 0, "fp32": 1, "bf16": 2}
VARIANT = {"additive": 0, "balanced": 1, "one_level": 2, "coarse_only": 3}
WEIGHTING = {"none": 0, "omega": 1}
KERNEL_CLASSES = ["keygen", "sort", "assemble", "potrf", "trsm", "syrk", "coarse_assemble",
                  "stencil", "update", "restrict", "trsv_fwd", "trsv_bwd", "prolong", "vector",
                  "grad", "coarse_factor", "pcg_vector"]

# Every exported function the header declares (checked by a CPU test).
EXPORTS = [
    "sfcdd_default_options", "sfcdd_setup", "sfcdd_setup_ex", "sfcdd_solve", "sfcdd_solve_host",
    "sfcdd_solve_backward", "sfcdd_apply_operator", "sfcdd_apply_precond", "sfcdd_get_info",
    "sfcdd_get_curve", "sfcdd_get_partition", "sfcdd_get_coarse_matrix", "sfcdd_get_local_matrix",
    "sfcdd_set_profiling", "sfcdd_get_kernel_stats", "sfcdd_kernel_work", "sfcdd_destroy",
    "sfcdd_status_string", "sfcdd_curve_order_noalloc", "sfcdd_batch_setup",
    "sfcdd_batch_offsets", "sfcdd_batch_solve", "sfcdd_batch_info", "sfcdd_batch_destroy",
    "sfcdd_estimate_spectrum", "sfcdd_richardson", "sfcdd_solve_homogeneous",
    "sfcdd_batch_setup_each", "sfcdd_batch_combine", "sfcdd_autotune", "sfcdd_batch_autotune",
    "sfcdd_selftest", "sfcdd_measure_fp64_rate",
]


class Tuning(C.Structure):
    _fields_ = [("slabs_local", C.c_int), ("slabs_coarse", C.c_int), ("apply_ms", C.c_double),
                ("candidates", C.c_int)]


class Options(C.Structure):
    _fields_ = [("coeffs", C.POINTER(C.c_double)), ("q", C.c_int), ("variant", C.c_int),
                ("weighting", C.c_int), ("precision", C.c_int), ("flexible", C.c_int),
                ("stream", C.c_void_p), ("profile", C.c_int), ("local_order", C.c_int),
                ("slabs_local", C.c_int), ("slabs_coarse", C.c_int), ("tensor_cores", C.c_int),
                ("coarse_block", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("status", C.c_int), ("fail_index", C.c_int),
                ("reserved", C.c_int), ("rel_res", C.c_double), ("true_rel_res", C.c_double),
                ("setup_ms", C.c_double), ("solve_ms", C.c_double)]


class Info(C.Structure):
    _fields_ = [("N", C.c_longlong), ("N0", C.c_longlong), ("d", C.c_int), ("P", C.c_int),
                ("q", C.c_int), ("nbits", C.c_int), ("tile", C.c_int), ("precision", C.c_int),
                ("variant", C.c_int), ("weighting", C.c_int), ("flexible", C.c_int),
                ("factor_bytes", C.c_longlong), ("coarse_bytes", C.c_longlong),
                ("setup_ms", C.c_double)]


class SfcddError(RuntimeError):
    def __init__(self, fn, code, detail=""):
        self.code = code
        super().__init__(f"{fn} failed: {STATUS.get(code, code)} ({code}) {detail}".strip())


_lib = None


def lib() -> C.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"{LIB_PATH} is missing: build it with paper_2110_11211_gb300.build.build() "
            "(there is no fallback implementation)")
    L = C.CDLL(LIB_PATH)
    H = C.c_void_p
    P = C.c_void_p
    L.sfcdd_default_options.argtypes = [C.POINTER(Options)]
    L.sfcdd_default_options.restype = None
    L.sfcdd_setup.argtypes = [C.POINTER(C.c_int), C.c_int, C.c_int, C.c_double, C.POINTER(H)]
    L.sfcdd_setup_ex.argtypes = [C.POINTER(C.c_int), C.c_int, C.c_int, C.c_double,
                                 C.POINTER(Options), C.POINTER(H)]
    L.sfcdd_solve.argtypes = [H, P, P, C.c_double, C.c_int, C.POINTER(Stats)]
    L.sfcdd_solve_host.argtypes = [H, P, P, C.c_double, C.c_int, C.POINTER(Stats)]
    L.sfcdd_solve_backward.argtypes = [H, P, P, P, C.POINTER(C.c_double), C.c_double, C.c_int,
                                       C.POINTER(Stats)]
    L.sfcdd_apply_operator.argtypes = [H, P, P, C.c_int]
    L.sfcdd_apply_precond.argtypes = [H, P, P, C.c_int]
    L.sfcdd_get_info.argtypes = [H, C.POINTER(Info)]
    L.sfcdd_get_curve.argtypes = [H, P, P]
    L.sfcdd_get_partition.argtypes = [H, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                      C.POINTER(C.c_double)]
    L.sfcdd_get_coarse_matrix.argtypes = [H, P]
    L.sfcdd_get_local_matrix.argtypes = [H, C.c_int, P]
    L.sfcdd_set_profiling.argtypes = [H, C.c_int]
    L.sfcdd_get_kernel_stats.argtypes = [H, C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.c_int]
    L.sfcdd_kernel_work.argtypes = [H, C.c_int]
    L.sfcdd_kernel_work.restype = C.c_double
    L.sfcdd_destroy.argtypes = [H]
    L.sfcdd_status_string.argtypes = [C.c_int]
    L.sfcdd_status_string.restype = C.c_char_p
    L.sfcdd_curve_order_noalloc.argtypes = [C.POINTER(C.c_int), C.c_int, P, P, C.c_void_p]
    L.sfcdd_batch_setup.argtypes = [C.POINTER(C.c_int), C.c_int, C.c_int, C.c_int, C.c_double,
                                    C.POINTER(Options), C.POINTER(H)]
    L.sfcdd_batch_setup_each.argtypes = [C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int,
                                         C.c_int, C.c_double, C.POINTER(Options), C.POINTER(H)]
    L.sfcdd_batch_combine.argtypes = [H, C.POINTER(C.c_double), P, P, C.c_longlong, P]
    L.sfcdd_autotune.argtypes = [H, C.c_int, C.POINTER(Tuning)]
    L.sfcdd_selftest.argtypes = [H, C.c_int, C.POINTER(C.c_int)]
    L.sfcdd_batch_autotune.argtypes = [H, C.c_int, C.POINTER(Tuning)]
    L.sfcdd_batch_offsets.argtypes = [H, C.POINTER(C.c_longlong)]
    L.sfcdd_batch_solve.argtypes = [H, P, P, C.c_double, C.c_int, C.POINTER(Stats),
                                    C.POINTER(Stats)]
    L.sfcdd_batch_info.argtypes = [H, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                   C.POINTER(C.c_double)]
    L.sfcdd_batch_destroy.argtypes = [H]
    L.sfcdd_estimate_spectrum.argtypes = [H, P, C.c_int, C.POINTER(C.c_double),
                                          C.POINTER(C.c_double)]
    L.sfcdd_richardson.argtypes = [H, P, P, C.c_double, C.c_double, C.c_int, C.POINTER(Stats)]
    L.sfcdd_solve_homogeneous.argtypes = [H, P, P, C.c_int, C.c_double, C.c_double, C.c_int,
                                          C.POINTER(Stats)]
    L.sfcdd_measure_fp64_rate.argtypes = [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                          C.c_void_p]
    for name in EXPORTS:
        if name not in ("sfcdd_default_options", "sfcdd_kernel_work", "sfcdd_status_string"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def check(fn: str, rc: int, detail: str = "") -> None:
    if rc != SFCDD_OK:
        raise SfcddError(fn, rc, detail)
