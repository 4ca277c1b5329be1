"""ctypes declarations of the C ABI in include/hps.h (argument marshalling only)."""

import ctypes
import os
import re

from . import build as _build

HPS_OK = 0
HPS_EINVAL = -1
HPS_ENOMEM = -2
HPS_ECUDA = -3
HPS_ENOCONV = -4
HPS_EBREAKDOWN = -5
HPS_ETIMEOUT = -6
HPS_C128 = 0
HPS_C64 = 1
HPS_C64_H16 = 2
HPS_FORM_FP64 = 1
HPS_FORM_MIXED = 2
HPS_SOLVE_NO_PRECOND = 16
HPS_SOLVE_X0 = 32
HPS_SOLVE_NO_GRAPH = 64
HPS_SOLVE_CGS2 = 128
HPS_INJECT_NONE = 0
HPS_INJECT_SKIP_ARRIVAL = 1
HPS_PRECOND_NOALLOC_MAX_BYTES = 16 << 20
HPS_EXPORT_R = 0
HPS_EXPORT_H = 1
HPS_EXPORT_LAMBDA = 2
HPS_EXPORT_KC = 3
HPS_EXPORT_B = 4

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "hps.h")


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("p", ctypes.c_int), ("q", ctypes.c_int)]


class Options(ctypes.Structure):
    _fields_ = [("forms", ctypes.c_int), ("restart", ctypes.c_int), ("cluster", ctypes.c_int),
                ("maxit", ctypes.c_int), ("max_rhs", ctypes.c_int), ("hbm_budget", ctypes.c_size_t),
                ("device", ctypes.c_int), ("precond_fp16", ctypes.c_int), ("tc_apply", ctypes.c_int),
                ("lean", ctypes.c_int), ("lambda_bin", ctypes.c_double), ("autotune", ctypes.c_int),
                ("full_system", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("cycles", ctypes.c_int), ("converged", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("seconds", ctypes.c_double), ("reorth_steps", ctypes.c_int)]


class LaunchShapes(ctypes.Structure):
    _fields_ = [("apply_rows_per_warp", (ctypes.c_int * 4) * 2), ("apply_ctas_per_sm", (ctypes.c_int * 4) * 2),
                ("stage_k_rows_per_warp", ctypes.c_int * 4), ("stage_k_ctas_per_sm", ctypes.c_int * 4),
                ("tuned", ctypes.c_int)]


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("ms", ctypes.c_double * 8), ("count", ctypes.c_longlong * 8)]


PHASES = ["apply", "precond_b", "precond_k", "arnoldi", "residual", "rhs", "update"]

_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)

SIGNATURES = {
    "hps_default_options": (None, [ctypes.POINTER(Options)]),
    "hps_nodes": (ctypes.c_int, [ctypes.POINTER(Grid), _P, _P, _P]),
    "hps_setup": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_double, ctypes.c_double, _P,
                                 ctypes.POINTER(Options), ctypes.POINTER(_P)]),
    "hps_apply": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int, _P]),
    "hps_precond": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int, _P]),
    "hps_precond_noalloc": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int, _P]),
    "hps_rhs": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, _P]),
    "hps_gmres_solve": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int, ctypes.c_double, _P,
                                       ctypes.POINTER(SolveInfo), _P]),
    "hps_recover": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, _P, _P]),
    "hps_export": (ctypes.c_longlong, [_P, ctypes.c_int, ctypes.c_int, _P]),
    "hps_import_map": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P]),
    "hps_test_inject": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_longlong]),
    "hps_get_launch_shapes": (ctypes.c_int, [_P, ctypes.POINTER(LaunchShapes)]),
    "hps_full_apply": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int, _P]),
    "hps_full_precond": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int, _P]),
    "hps_full_solve": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int, ctypes.c_double, _P,
                                      ctypes.POINTER(SolveInfo), _P]),
    "hps_precond_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int)]),
    "hps_memory_bytes": (ctypes.c_size_t, [_P]),
    "hps_setup_bytes": (ctypes.c_size_t, [ctypes.POINTER(Grid), ctypes.POINTER(Options), ctypes.c_int]),
    "hps_axis_eig": (ctypes.c_int, [ctypes.c_int, _P, _P, _P, _P]),
    "hps_plan_blocks": (ctypes.c_int, [ctypes.POINTER(Grid), _P, _P, _P, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "hps_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "hps_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(Profile), ctypes.c_int]),
    "hps_destroy": (ctypes.c_int, [_P]),
    "hps_last_error": (ctypes.c_char_p, []),
}

_lib = None


def header_functions(path=HEADER):
    """Names of the functions declared in include/hps.h."""
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hps_[a-z_0-9]+)\s*\(", src)))


def load(path=None, build=True):
    """Load libhps.so (building it in-tree first when sources changed)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    if path is None:
        path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; build it with __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path == _build.LIB or _lib is None:
        _lib = lib
    return lib


class HPSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"HPS error {code}: {msg}")
        self.code = code


def check(rc):
    if rc < 0:
        raise HPSError(rc, load().hps_last_error().decode())
    return rc
