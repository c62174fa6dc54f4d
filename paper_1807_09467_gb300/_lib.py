"""ctypes declarations of librgmres (include/rgmres.h).

The library is the in-tree build at ``paper_1807_09467_gb300/_build/librgmres.so``.
There is no fallback: if it is missing or cannot be loaded, loading raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librgmres.so")

RGM_OK = 0
RGM_W_NOT_CONVERGED = 1
RGM_W_SINGULAR_COARSE = 2
RGM_E_ARG = -1
RGM_E_OOM = -2
RGM_E_CUDA = -3
RGM_E_STATE = -4
RGM_E_TIMEOUT = -5
RGM_DEVICE_PTRS = 1
RGM_BATCH_COOP = 2
RGM_ZERO_GUESS = 4
RGM_NOALLOC_MAX_ROWS = 4096 * 2048

PLAIN, DEFLATED, AUGMENTED, GUESS = 0, 1, 2, 3
FP64, FP32_IR = 0, 1


class RgmConfig(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int), ("k", C.c_int), ("window", C.c_int),
                ("svd_interval", C.c_int), ("select_smallest", C.c_int), ("mode", C.c_int),
                ("precision", C.c_int), ("start_r", C.c_int), ("maxit", C.c_int),
                ("inner_cycles", C.c_int), ("max_refinements", C.c_int), ("launch_policy", C.c_int),
                ("proj", C.c_int), ("guess", C.c_int), ("precond", C.c_int), ("tiles_per_block", C.c_int),
                ("rtol", C.c_double),
                ("inner_rtol", C.c_double), ("rel_drop", C.c_double), ("cuda_stream", C.c_void_p)]


class RgmStats(C.Structure):
    _fields_ = [("iters", C.c_int), ("cycles", C.c_int), ("refinements", C.c_int),
                ("k_used", C.c_int), ("status", C.c_int), ("true_relres", C.c_double)]


class RgmKernelProf(C.Structure):
    _fields_ = [("ms", C.c_double), ("launches", C.c_int64), ("flops", C.c_double),
                ("bytes", C.c_double), ("units", C.c_double), ("step_bytes", C.c_double)]


PROF_KINDS = ["arnoldi_spmv_dots", "arnoldi_cgs1_axpy_dots", "arnoldi_cgs2_axpy_norm", "other_vector",
              "gram", "small", "arnoldi_cycle", "window_svd", "coarse_setup", "operator_values"]

_lib = None
_lock = threading.Lock()

# name -> (restype, argtypes)
_SIGS = {
    "rgm_config_default": (C.c_int, [C.POINTER(RgmConfig)]),
    "rgm_solver_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(RgmConfig)]),
    "rgm_solver_destroy": (C.c_int, [C.c_void_p]),
    "rgm_set_operator_csr": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_int]),
    "rgm_set_operator_values": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "rgm_set_operator_sell": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_int]),
    "rgm_set_recycle_space": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int64, C.c_int]),
    "rgm_get_recycle_space": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int),
                                        C.c_int]),
    "rgm_export_state": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_size_t)]),
    "rgm_import_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "rgm_last_error": (C.c_char_p, []),
    "rgm_wait_selftest": (C.c_int, [C.c_int64, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "rgm_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(RgmStats)]),
    "rgm_batch_solve": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                  C.c_void_p]),
    "rgm_batch_plan": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                 C.c_void_p, C.c_void_p, C.c_void_p]),
    "rgm_update_recycle_svd": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "rgm_get_singular_values": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]),
    "rgm_reset_recycling": (C.c_int, [C.c_void_p]),
    "rgm_spmv": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "rgm_status_string": (C.c_char_p, [C.c_int]),
    "rgm_solver_device_bytes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "rgm_fe_device_bytes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "rgm_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "rgm_profile_read": (C.c_int, [C.c_void_p, C.POINTER(RgmKernelProf), C.c_int,
                                   C.POINTER(C.c_int64)]),
    "rgm_residual_noalloc": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rgm_fe_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_double, C.c_double,
                                C.c_double, C.c_double, C.c_void_p]),
    "rgm_fe_destroy": (C.c_int, [C.c_void_p]),
    "rgm_fe_sizes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "rgm_fe_pattern": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "rgm_fe_assemble": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "rgm_fe_initial_field": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "rgm_fe_set_velocity": (C.c_int, [C.c_void_p, C.c_int]),
    "rgm_fe_set_forcing": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_double, C.c_int]),
    "rgm_fe_time_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(RgmStats)]),
}

EXPORTED = sorted(_SIGS)


def load():
    """Load librgmres.so (raises OSError / RuntimeError if it is not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"librgmres is not built ({LIB_PATH} missing): run "
                    "`python -c 'import __graft_entry__ as g; g.build()'` first")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
        return _lib


class RgmError(RuntimeError):
    def __init__(self, code, what):
        L = load()
        msg = L.rgm_status_string(code).decode()
        if code in (RGM_E_CUDA, RGM_E_OOM):
            detail = L.rgm_last_error().decode()
            if detail:
                msg += f": {detail}"
        super().__init__(f"{what}: {msg} ({code})")
        self.code = code


def check(code, what):
    if code < 0:
        raise RgmError(code, what)
    return code
