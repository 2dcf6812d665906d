"""ctypes declarations of the C ABI in include/pppc.h.

Only argument marshalling lives here: every floating-point step of the method
runs in the CUDA kernels of libpppc.so.  Loading fails loudly when the library
has not been built; there is no fallback path.
"""

from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int32, c_int64, c_uint8, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpppc.so")

PPPC_OK = 0
STATUS_NAMES = {
    0: "PPPC_OK", 1: "PPPC_ERR_INVALID_ARG", 2: "PPPC_ERR_CUDA", 3: "PPPC_ERR_STATE",
    4: "PPPC_ERR_NEWTON", 5: "PPPC_ERR_LINEAR", 6: "PPPC_ERR_BREAKDOWN", 7: "PPPC_ERR_NAN",
    8: "PPPC_ERR_TIMEOUT", 9: "PPPC_ERR_NOT_CONVERGED", 10: "PPPC_ERR_UNSUPPORTED",
    11: "PPPC_ERR_NOMEM",
}
PPPC_FP64, PPPC_MIXED = 0, 1
COARSE_LIN = {"avg_jacobian": 0, "avg_chord": 1, "zero_field": 2}
METHODS = {"pppc": 0, "ppic": 1}
COARSE_AT = {"U": 0, "F": 1}
NU_LINEAR, NU_BRAUER = 0, 1

ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, ctypes.c_size_t, c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_void_p)


class pppc_config(ctypes.Structure):
    _fields_ = [
        ("T", c_double), ("N", c_int32), ("n_fine", c_int32), ("precision", c_int32),
        ("coarse_lin", c_int32), ("tol_newton", c_double), ("max_newton", c_int32),
        ("tol_lin", c_double), ("max_lin", c_int32), ("tol_coarse", c_double),
        ("max_coarse", c_int32), ("stream", c_void_p), ("alloc", c_void_p),
        ("free_fn", c_void_p), ("alloc_ctx", c_void_p), ("eta0", c_double), ("predictor", c_int32),
        ("method", c_int32), ("coarse_at", c_int32), ("newton_schedule", c_int32), ("precond", c_int32),
        ("lane_team", c_int32),
    ]


class pppc_material(ctypes.Structure):
    _fields_ = [
        ("sigma", c_double), ("nu_model", c_int32), ("nu", c_double),
        ("k1", c_double), ("k2", c_double), ("k3", c_double), ("is_source", c_int32), ("bmax", c_double),
    ]


class pppc_stats(ctypes.Structure):
    _fields_ = [
        ("newton_iters", c_int64), ("pcg_iters", c_int64), ("cocg_iters", c_int64),
        ("fine_steps", c_int64), ("pppc_iters", c_int32), ("rel_res", c_double),
        ("fine_ms", c_double), ("coarse_ms", c_double), ("launches", c_int64), ("backtracks", c_int64),
        ("pcg_lane_rounds", c_int64), ("pcg_lane_iters", c_int64), ("newton_lane_rounds", c_int64),
        ("graph_launches", c_int64),
    ]


class pppc_fine_plan_info(ctypes.Structure):
    _fields_ = [("lanes_per_team", c_int32), ("teams", c_int32), ("threads_per_row", c_int32),
                ("blocks_min", c_int32), ("blocks_max", c_int32), ("n_candidates", c_int32),
                ("candidate_lanes", c_int32 * 16), ("candidate_ms", c_double * 16), ("amg_levels", c_int32),
                ("amg_rows", c_int32 * 10)]


class pppc_mesh_counts(ctypes.Structure):
    _fields_ = [("ndof", c_int64), ("nnz", c_int64), ("special_rows", c_int64),
                ("special_entries", c_int64), ("nonlinear_elems", c_int64)]


class pppc_adjoint_result(ctypes.Structure):
    _fields_ = [("loss", c_double), ("grad", c_double * 4), ("iterations", c_int32), ("rel_res", c_double),
                ("forward_rel_res", c_double)]


class pppc_batch_stats(ctypes.Structure):
    _fields_ = [("iterations", c_int32), ("retunes", c_int32), ("graph_launches", c_int64),
                ("kernel_launches", c_int64), ("fine_dof_steps", c_int64), ("fine_ms", c_double),
                ("coarse_ms", c_double)]


_DPTR = POINTER(c_double)
_IPTR = POINTER(c_int32)

# name -> (restype, argtypes); the names and order follow include/pppc.h
SIGNATURES = {
    "pppc_config_default": (None, [POINTER(pppc_config)]),
    "pppc_create": (c_int32, [POINTER(pppc_config), POINTER(c_void_p)]),
    "pppc_destroy": (None, [c_void_p]),
    "pppc_set_mesh": (c_int32, [c_void_p, c_int32, c_void_p, c_int32, c_void_p, c_void_p, c_void_p,
                                c_int32, POINTER(pppc_material)]),
    "pppc_set_source": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "pppc_set_state": (c_int32, [c_void_p, c_void_p, c_int32]),
    "pppc_get_state": (c_int32, [c_void_p, c_void_p, c_int32]),
    "pppc_propagate_fine": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32]),
    "pppc_propagate_fine_window": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32]),
    "pppc_coarse_update": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, _DPTR, c_int32]),
    "pppc_iterate": (c_int32, [c_void_p, _DPTR]),
    "pppc_solve_periodic": (c_int32, [c_void_p, c_double, c_int32, _IPTR, _DPTR]),
    "pppc_get_stats": (c_int32, [c_void_p, POINTER(pppc_stats)]),
    "pppc_get_fine_plan": (c_int32, [c_void_p, POINTER(pppc_fine_plan_info)]),
    "pppc_set_trace": (c_int32, [c_void_p, c_int32]),
    "pppc_get_trace": (c_int32, [c_void_p, c_void_p, c_int32, _IPTR]),
    "pppc_ndof": (c_int32, [c_void_p]),
    "pppc_get_mesh_counts": (c_int32, [c_void_p, POINTER(pppc_mesh_counts)]),
    "pppc_last_error": (c_char_p, [c_void_p]),
    "pppc_status_string": (c_char_p, [c_int32]),
    "pppc_harmonic_solve_noalloc": (c_int32, [c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_int32,
                                              c_void_p, c_void_p, c_double, c_int32, c_void_p, _IPTR]),
    "pppc_selftest_wait_timeout": (c_int32, [c_void_p]),
    "pppc_binary_version": (c_int32, [_IPTR]),
    "pppc_adjoint": (c_int32, [c_void_p, c_int32, c_double, c_int32, POINTER(pppc_adjoint_result)]),
    "pppc_batch_create": (c_int32, [POINTER(c_void_p), c_int32, c_int32, POINTER(c_void_p)]),
    "pppc_batch_destroy": (None, [c_void_p]),
    "pppc_batch_iterate": (c_int32, [c_void_p, _DPTR]),
    "pppc_batch_solve_periodic": (c_int32, [c_void_p, c_double, c_int32, _IPTR, _DPTR]),
    "pppc_batch_get_stats": (c_int32, [c_void_p, POINTER(pppc_batch_stats)]),
    "pppc_batch_get_teams": (c_int32, [c_void_p, _IPTR, _IPTR]),
    "pppc_batch_get_lanes": (c_int32, [c_void_p, _IPTR, _IPTR]),
    "pppc_batch_last_error": (c_char_p, [c_void_p]),
    "pppc_batch_plan": (c_int32, [_DPTR, _IPTR, _IPTR, c_int32, c_int32, _IPTR, _DPTR]),
}

_lib = None


def load(path: str | None = None):
    """Load libpppc.so (built by ``paper_1905_13076_gb300.build``)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"{p} is missing: build it with `python -m paper_1905_13076_gb300.build` "
                          "(the library has no CPU fallback)")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


class PPPCError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message


def check(status: int, handle=None):
    if status != PPPC_OK:
        lib = load()
        msg = lib.pppc_last_error(handle)
        raise PPPCError(status, msg.decode() if msg else "")


def check_batch(status: int, batch=None):
    if status != PPPC_OK:
        lib = load()
        msg = lib.pppc_batch_last_error(batch)
        raise PPPCError(status, msg.decode() if msg else "")
