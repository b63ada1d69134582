"""ctypes loader of libstfdm.so and the C structs of include/stfdm.h.

Fails loudly when the library is missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_int = ctypes.c_int
c_double = ctypes.c_double
c_void_p = ctypes.c_void_p
c_char_p = ctypes.c_char_p

ST_OK = 0
ST_ERR_ARG = -1
ST_ERR_OOM = -2
ST_ERR_CUDA = -3
ST_ERR_ILL_CONDITIONED = -4
ST_ERR_ZERO_PIVOT = -5
ST_ERR_NOT_CONVERGED = -6
ST_ERR_TIMEOUT = -7
ST_ERR_UNSUPPORTED = -8

ST_SPATIAL_AUTO = 0
ST_SPATIAL_BANDED = 1
ST_SPATIAL_MULTIFRONTAL = 2

ST_FP64 = 0
ST_FP32 = 1
ST_MIXED = 2

ST_REFINE_GMRES = 0
ST_REFINE_CLASSIC = 1

ST_EXACT_C1 = 0
ST_EXACT_PAPER = 1

ST_XFORM_Y = 0
ST_XFORM_X = 1
ST_XFORM_XT = 2
ST_XFORM_YT = 3


class st_setup_opts(ctypes.Structure):
    _fields_ = [("kappa_max", c_double), ("device", c_int), ("host_threads", c_int), ("spatial_solver", c_int)]


class st_solve_opts(ctypes.Structure):
    _fields_ = [("precision", c_int), ("tol", c_double), ("max_sweeps", c_int), ("keep_factors", c_int),
                ("fixed_sweeps", c_int), ("method", c_int), ("err_tol", c_double)]


class st_solve_info(ctypes.Structure):
    _fields_ = [("sweeps", c_int), ("factors_kept", c_int), ("rel_residual", c_double),
                ("residual_history", c_double * 16), ("kappa_x", c_double), ("min_neg_im_shift", c_double),
                ("setup_seconds", c_double), ("tensor_cores", c_int), ("kernel_launches", c_int),
                ("restart", c_int), ("rel_error_estimate", c_double), ("kept_systems", c_int),
                ("reorth_steps", c_int)]


class st_batch_opts(ctypes.Structure):
    _fields_ = [("tol", c_double), ("max_sweeps", c_int), ("restart", c_int), ("no_graph", c_int),
                ("no_tune", c_int), ("no_keep", c_int)]


class st_batch_stats(ctypes.Structure):
    _fields_ = [("count", c_int), ("items", c_int), ("restart", c_int), ("xform_tile_m", c_int),
                ("xform_tile_n", c_int), ("solve_ctas_per_sm", c_int), ("solve_grid", c_int),
                ("graph_nodes", c_int), ("cycles", c_int), ("tuned", c_int), ("tune_seconds", c_double),
                ("unknowns", ctypes.c_longlong), ("workspace_bytes", ctypes.c_ulonglong),
                ("kept_problems", c_int), ("kept_factor_bytes", ctypes.c_ulonglong)]


# name -> (restype, argtypes); every entry point declared in include/stfdm.h
SIGNATURES = {
    "st_status_string": (c_char_p, [c_int]),
    "st_last_error_message": (c_char_p, []),
    "st_abi_version": (c_int, []),
    "st_assemble_time": (c_int, [c_int, c_int, ctypes.POINTER(c_double), ctypes.POINTER(c_void_p)]),
    "st_time_get": (c_int, [c_void_p, ctypes.POINTER(c_int), c_void_p, c_void_p, c_void_p, c_void_p]),
    "st_assemble_space": (c_int, [c_int, c_double, c_double, ctypes.POINTER(c_void_p)]),
    "st_space_get": (c_int, [c_void_p, ctypes.POINTER(c_int), ctypes.POINTER(c_int), c_void_p]),
    "st_time_decompose": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_double)]),
    "st_fdm_setup": (c_int, [c_void_p, c_void_p, ctypes.POINTER(st_setup_opts), ctypes.POINTER(c_void_p)]),
    "st_fdm_get": (c_int, [c_void_p, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                           ctypes.POINTER(c_double), ctypes.POINTER(c_double)]),
    "st_fdm_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, ctypes.POINTER(st_solve_opts),
                             ctypes.POINTER(st_solve_info), c_void_p]),
    "st_residual": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_double), c_void_p]),
    "st_adjoint_solve": (c_int, [c_void_p, c_void_p, c_void_p, ctypes.POINTER(st_solve_opts),
                                 ctypes.POINTER(st_solve_info), c_void_p]),
    "st_adjoint_lift": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "st_fdm_solve_batched": (c_int, [ctypes.POINTER(c_void_p), c_int, ctypes.POINTER(c_void_p),
                                     ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                     ctypes.POINTER(st_solve_opts), ctypes.POINTER(st_solve_info), c_void_p]),
    "st_batch_create": (c_int, [ctypes.POINTER(c_void_p), c_int, ctypes.POINTER(st_batch_opts),
                                ctypes.POINTER(c_void_p)]),
    "st_batch_solve": (c_int, [c_void_p, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                               ctypes.POINTER(st_solve_info), c_void_p]),
    "st_batch_spatial_solve": (c_int, [c_void_p, c_void_p]),
    "st_batch_spatial_get": (c_int, [c_void_p, c_int, c_void_p, c_int, c_void_p]),
    "st_batch_stats_get": (c_int, [c_void_p, ctypes.POINTER(st_batch_stats)]),
    "st_destroy_batch": (None, [c_void_p]),
    "st_time_transform": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "st_spatial_solve": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "st_load_nodal": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "st_error_norms": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_int, c_int, ctypes.POINTER(c_double), c_void_p]),
    "st_load_quadrature": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p]),
    "st_residual_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "st_set_wait_probe": (c_int, [c_void_p, c_double]),
    "st_bs_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "st_spatial_factor": (c_int, [c_void_p, c_int, c_void_p]),
    "st_spatial_substitute": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "st_assemble_mesh": (c_int, [c_int, c_int, c_int, c_void_p, c_int, c_void_p, c_void_p]),
    "st_space_get_mesh": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                  c_void_p, c_void_p]),
    "st_space_mf_plan": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                 c_void_p, c_void_p, c_void_p, c_void_p]),
    "st_destroy_time": (None, [c_void_p]),
    "st_destroy_space": (None, [c_void_p]),
    "st_destroy_fdm": (None, [c_void_p]),
}

_LIB = None


def lib():
    """The loaded library (built in-tree by __graft_entry__.build())."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(
                f"stfdm CUDA library not found at {path}: run __graft_entry__.build() "
                "(there is no CPU fallback)")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


class StfdmError(RuntimeError):
    info = None

    def __init__(self, status: int, where: str):
        L = lib()
        msg = L.st_last_error_message()
        super().__init__(f"{where}: {L.st_status_string(status).decode()} ({status}): "
                         f"{msg.decode() if msg else ''}")
        self.status = status


def check(status: int, where: str):
    if status != ST_OK:
        raise StfdmError(status, where)
