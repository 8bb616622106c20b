"""ctypes view of the C ABI in include/rexi.h (argument marshalling only).

Loading fails loudly when librexi.so is missing: there is no fallback path.
"""

from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# REXI_DEBUG=1 selects the build with index checks of the Lanczos kernel
DEBUG_LIB_PATH = os.path.join(HERE, "librexi_debug.so")
LIB_PATH = DEBUG_LIB_PATH if os.environ.get("REXI_DEBUG") == "1" else os.path.join(HERE, "librexi.so")

REXI_OK = 0
REXI_EINVAL = -1
REXI_ENOMEM = -2
REXI_ECUDA = -3
REXI_ENOCONV = -4
REXI_ETIMEOUT = -5
REXI_EPLAN = -6
REXI_EBOUNDS = -7
REXI_WACCURACY = 1
REXI_FP64 = 0
REXI_MIXED = 1
REXI_DF64 = 2
REXI_MAX_POLES = 256
REXI_MAX_RESTART = 64
REXI_MAX_RESTART_FULL = 31
REXI_MAX_KRYLOV = 512

# sites of the index checks of the debug build (csrc/lanczos.h)
LZ_SITES = {1: "smem", 2: "stage", 3: "stage_src", 4: "ring", 5: "basis", 6: "stencil", 7: "wt", 8: "part",
            9: "rows", 10: "y", 11: "state"}


class Grid(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("hbar", C.c_double), ("mass", C.c_double)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("restart_m", C.c_int), ("max_iters", C.c_int),
                ("tol", C.c_double), ("inner_tol", C.c_double), ("R1", C.c_double),
                ("eps_target", C.c_double), ("allow_substeps", C.c_int), ("stabilize_eps", C.c_double),
                ("want_backward", C.c_int), ("device", C.c_int), ("shared_first_cycle", C.c_int),
                ("ortho", C.c_int), ("window", C.c_int)]


class PlanInfo(C.Structure):
    _fields_ = [("K", C.c_int), ("n_sub", C.c_int), ("n_total", C.c_int), ("restart_m", C.c_int),
                ("precision", C.c_int), ("dt", C.c_double), ("tau", C.c_double), ("R1", C.c_double),
                ("sigma_K1", C.c_double), ("E_min", C.c_double), ("E_max", C.c_double), ("c", C.c_double),
                ("W", C.c_double), ("amplification", C.c_double), ("tol", C.c_double),
                ("min_re_sigma", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("status", C.c_int), ("n_sub", C.c_int), ("max_iters_seen", C.c_int),
                ("total_iters", C.c_int), ("total_cycles", C.c_int),
                ("iters", C.c_int * REXI_MAX_POLES), ("cycles", C.c_int * REXI_MAX_POLES),
                ("iters_sq", C.c_int * REXI_MAX_POLES), ("resid", C.c_double * REXI_MAX_POLES),
                ("bytes", C.c_double), ("flops64", C.c_double), ("ops32", C.c_double)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)

SIGNATURES = {
    "rexi_options_default": (C.c_int, [C.POINTER(Options)]),
    "rexi_plan_create": (C.c_int, [C.POINTER(_P), C.POINTER(Grid), _D, C.c_double, C.c_int,
                                   C.POINTER(Options)]),
    "rexi_plan_destroy": (None, [_P]),
    "rexi_plan_get_info": (C.c_int, [_P, C.POINTER(PlanInfo)]),
    "rexi_plan_poles": (C.c_int, [_P, _D, _D, _D, C.POINTER(C.c_int)]),
    "rexi_plan_fcf": (C.c_int, [_P, _D, _D]),
    "rexi_fcf": (C.c_int, [C.c_int, C.c_double, C.c_double, _D, _D, _D, _D, _D, _D]),
    "rexi_plan_set_potential": (C.c_int, [_P, _P, C.c_int, _P]),
    "rexi_step": (C.c_int, [_P, _P, _P, _P, C.POINTER(Stats)]),
    "rexi_step_host": (C.c_int, [_P, _P, _P, _P, C.POINTER(Stats)]),
    "rexi_step_batched": (C.c_int, [C.POINTER(_P), C.c_int, C.POINTER(_P), C.POINTER(_P), _P,
                                    C.POINTER(Stats)]),
    "rexi_step_backward": (C.c_int, [_P, _P, _P, _P, _P, _P, C.POINTER(Stats)]),
    "rexi_apply_poles": (C.c_int, [_P, _P, _P, _P]),
    "rexi_solve_poles": (C.c_int, [_P, _P, _P, _P, C.POINTER(Stats)]),
    "rexi_pole_sum": (C.c_int, [_P, _P, _P, _P, _P]),
    "rexi_plan_last_status": (C.c_int, [_P]),
    "rexi_plan_last_launches": (C.c_int, [_P]),
    "rexi_debug_checks": (C.c_int, []),
    "rexi_plan_debug_record": (C.c_int, [_P, C.POINTER(C.c_longlong)]),
    "rexi_plan_debug_trip": (C.c_int, [_P, C.c_int]),
    "rexi_plan_set_trace": (C.c_int, [_P, C.c_int]),
    "rexi_plan_set_tiles": (C.c_int, [_P, C.c_int, C.c_int, C.c_int]),
    "rexi_plan_set_timeout": (C.c_int, [_P, C.c_double]),
    "rexi_plan_read_trace": (C.c_int, [_P, C.POINTER(C.c_longlong), C.c_int]),
    "rexi_plan_set_cta_trace": (C.c_int, [_P, C.c_int]),
    "rexi_cheb_step": (C.c_int, [_P, _P, _P, C.c_double, _P, C.POINTER(C.c_int)]),
    "rexi_plan_last_work": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "rexi_plan_read_cta_trace": (C.c_int, [_P, C.POINTER(C.c_longlong), C.c_int, C.POINTER(C.c_int)]),
    "rexi_status_string": (C.c_char_p, [C.c_int]),
    "rexi_substep_static": (C.c_int, [C.POINTER(Grid), _P, C.c_double, C.c_double, C.c_int, _D, _D, _D,
                                      C.POINTER(Options), _P, _P, _P, C.POINTER(Stats)]),
}

_lib = None


class RexiError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        msg = status_string(code) if _lib is not None else str(code)
        super().__init__("%s%s (status %d)" % (where + ": " if where else "", msg, code))


def load(path=None):
    """Load librexi.so (once).  Raises if it is missing or incomplete."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("%s not found: build it with `python -m paper_1912_03312_gb300.build` "
                           "(no CPU fallback exists)" % p)
    lib = C.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(code):
    return load().rexi_status_string(int(code)).decode()


def check(code, where=""):
    if code < 0:
        raise RexiError(code, where)
    return code
