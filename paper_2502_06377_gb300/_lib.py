"""ctypes binding of libibmi.so (include/ibmi.h).

Argument marshalling only: every step of the inversion runs in the CUDA
library.  If the library has not been built the import fails loudly; there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libibmi.so")

# ibmi_status
IBMI_OK = 0
IBMI_ERR_INVALID_ARG = 1
IBMI_ERR_NOT_SPD = 2
IBMI_NOT_CONVERGED = 3
IBMI_ERR_NONFINITE = 4
IBMI_ERR_BUDGET = 5
IBMI_ERR_OOM = 6
IBMI_ERR_TIMEOUT = 7
IBMI_ERR_CUDA = 8
IBMI_NOT_READY = 9
IBMI_ERR_CANCELLED = 10
# ibmi_precision / stop rule / init
IBMI_FP64 = 0
IBMI_MIXED = 1
IBMI_STOP_RESID_F = 0
IBMI_STOP_PAPER_EST = 1
IBMI_INIT_IDENTITY = 0
IBMI_INIT_USER = 1
IBMI_INIT_SCHUR = 2


class ibmi_plan_desc(C.Structure):
    _fields_ = [
        ("p", C.c_int64), ("K", C.c_int32), ("h", C.c_int64),
        ("lo", C.POINTER(C.c_int64)), ("hi", C.POINTER(C.c_int64)),
        ("precision", C.c_int32), ("tol", C.c_double), ("max_sweeps", C.c_int32),
        ("stop_rule", C.c_int32), ("check_every", C.c_int32), ("ns_theta", C.c_double),
        ("ns_max", C.c_int32), ("init", C.c_int32),
    ]


class ibmi_result(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("sweeps", C.c_int32), ("ns_steps", C.c_int32),
        ("bad_block", C.c_int32), ("bad_pivot", C.c_int64), ("resid_f", C.c_double),
        ("paper_est", C.c_double), ("seconds", C.c_double), ("flops", C.c_double),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_P = C.c_void_p
_D = C.POINTER(C.c_double)

_SIGS = {
    "ibmi_plan_desc_init": (None, [C.POINTER(ibmi_plan_desc)]),
    "ibmi_plan": (C.c_int, [C.POINTER(ibmi_plan_desc), C.POINTER(_P)]),
    "ibmi_plan_destroy": (C.c_int, [_P]),
    "ibmi_plan_sets": (C.c_int, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "ibmi_invert": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int64, _P, C.POINTER(ibmi_result)]),
    "ibmi_invert_host": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int64, _P, C.POINTER(ibmi_result)]),
    "ibmi_invert_block_diag": (C.c_int, [_P, _P, C.c_int64, _P, _P, C.POINTER(ibmi_result)]),
    "ibmi_residual": (C.c_int, [_P, C.c_int64, _P, C.c_int64, C.c_int64, _P, _D]),
    "ibmi_residual_tc": (C.c_int, [_P, C.c_int64, _P, C.c_int64, C.c_int64, _P, _D]),
    "ibmi_residual_noalloc": (C.c_int, [_P, C.c_int64, _P, C.c_int64, C.c_int64, _P, _D]),
    "ibmi_selftest_wait_timeout": (C.c_int, [_P]),
    "ibmi_refine": (C.c_int, [_P, C.c_int64, _P, C.c_int64, C.c_int64, C.c_int32, C.c_double, C.c_int32, _P,
                              C.POINTER(ibmi_result)]),
    "ibmi_prof_enable": (None, [C.c_int]),
    "ibmi_prof_get": (C.c_int, [C.c_int32, C.POINTER(C.c_int64), _D, _D]),
    "ibmi_prof_get_alg": (C.c_int, [C.c_int32, _D]),
    "ibmi_launch_count": (C.c_int64, []),
    "ibmi_status_string": (C.c_char_p, [C.c_int]),
    "ibmi_last_error": (C.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Loads the CUDA library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


IBMI_ORDER_IDENTITY, IBMI_ORDER_XSORT, IBMI_ORDER_HILBERT, IBMI_ORDER_KD, IBMI_ORDER_REDBLACK = 0, 1, 2, 3, 4


class ibmi_tune_candidate(C.Structure):
    _fields_ = [
        ("order", C.c_int32), ("K", C.c_int32), ("h", C.c_int64), ("status", C.c_int32),
        ("sweeps", C.c_int32), ("ns_steps", C.c_int32), ("seconds", C.c_double), ("resid_f", C.c_double),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_SIGS.update({
    "ibmi_order_points": (C.c_int, [C.POINTER(C.c_double), C.c_int64, C.c_int32, C.c_int32,
                                    C.POINTER(C.c_int64)]),
    "ibmi_permute": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.POINTER(C.c_int64), C.c_int32, C.c_void_p,
                               C.c_int64, C.c_void_p]),
    "ibmi_tune": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.POINTER(C.POINTER(C.c_int64)), C.c_int32,
                            C.POINTER(ibmi_plan_desc), C.c_void_p, C.POINTER(ibmi_tune_candidate),
                            C.POINTER(ibmi_tune_candidate), C.c_int32, C.POINTER(C.c_int32)]),
})


class ibmi_batch_opts(C.Structure):
    _fields_ = [
        ("precision", C.c_int32), ("tol", C.c_double), ("max_sweeps", C.c_int32),
        ("ns_theta", C.c_double), ("ns_max", C.c_int32), ("workers", C.c_int32), ("autotune", C.c_int32),
        ("graphs", C.c_int32), ("device_batch", C.c_int32),
    ]


class ibmi_batch_stats(C.Structure):
    _fields_ = [
        ("device_matrices", C.c_int64), ("groups", C.c_int64), ("rounds_max", C.c_int64),
        ("rounds_total", C.c_int64), ("fallbacks", C.c_int64), ("seconds_groups", C.c_double),
        ("seconds_single", C.c_double),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_SIGS.update({
    "ibmi_batch_last_stats": (C.c_int, [C.POINTER(ibmi_batch_stats)]),
    "ibmi_batch_opts_init": (None, [C.POINTER(ibmi_batch_opts)]),
    "ibmi_plan_bytes": (C.c_size_t, [C.POINTER(ibmi_plan_desc)]),
    "ibmi_invert_batched": (C.c_int, [C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_void_p),
                                      C.POINTER(C.c_int64), C.POINTER(C.c_void_p), C.POINTER(C.c_int64),
                                      C.POINTER(ibmi_batch_opts), C.POINTER(ibmi_result)]),
    "ibmi_batch_release": (C.c_int, []),
    "ibmi_serve_create": (C.c_int, [C.c_size_t, C.POINTER(ibmi_batch_opts), C.POINTER(C.c_void_p)]),
    "ibmi_serve_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_double,
                                    C.POINTER(C.c_uint64)]),
    "ibmi_serve_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_int64, C.POINTER(ibmi_result)]),
    "ibmi_serve_cancel": (C.c_int, [C.c_void_p, C.c_uint64]),
    "ibmi_serve_stats": (C.c_int, [C.c_void_p, _D, _D, _D, C.POINTER(C.c_int64), C.POINTER(C.c_uint64)]),
    "ibmi_serve_stats_reset": (C.c_int, [C.c_void_p]),
    "ibmi_serve_destroy": (C.c_int, [C.c_void_p]),
})
