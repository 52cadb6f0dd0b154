"""ctypes binding of libstbem.so (the C ABI declared in include/stbem.h).

Argument marshalling only: every step of the computation runs in the CUDA
library. The library is loaded from the package's build directory; if it is
missing, loading fails loudly (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

BEM_OK = 0
STATUS = {0: "BEM_OK", 1: "BEM_ERR_INVALID_ARG", 2: "BEM_ERR_OUT_OF_MEMORY", 3: "BEM_ERR_CUDA",
          4: "BEM_ERR_NOT_CONVERGED", 5: "BEM_ERR_DEVICE_TIMEOUT", 6: "BEM_ERR_UNSUPPORTED",
          7: "BEM_ERR_BAD_MESH", 8: "BEM_ERR_INTERNAL", 9: "BEM_ERR_CANCELLED"}
PREC = {"fp64": 0, "mixed": 1}
TRIAL = {"p0": 0, "p1": 1}
DTYPE = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3}
DATA_SIN2_UNIFORM = 0
DATA_PULSE = 1

# every symbol include/stbem.h declares
EXPORTS = [
    "bem_context_create", "bem_context_destroy", "bem_last_error", "bem_version", "bem_alu_peaks",
    "bem_context_set_tuning", "bem_operator_tuning", "bem_selftest_bounded_wait",
    "bem_mesh_create", "bem_mesh_create_prisms", "bem_mesh_info", "bem_mesh_destroy",
    "bem_operator_create", "bem_operator_stats", "bem_operator_check", "bem_operator_work", "bem_operator_timings", "bem_operator_reassemble", "bem_operator_export_pattern", "bem_operator_pattern_rows",
    "bem_operator_export_dense", "bem_operator_entries", "bem_operator_destroy",
    "bem_rhs", "bem_rhs_points", "bem_rhs_from_samples", "bem_matvec", "bem_matvec_dtype", "bem_matvec_noalloc", "bem_solve", "bem_solve_refined", "bem_solve_device",
    "bem_solve_async", "bem_request_wait", "bem_request_cancel", "bem_request_destroy", "bem_inner_potentials",
    "bem_batch_create", "bem_batch_stats", "bem_batch_solve", "bem_batch_destroy",
    "bem_server_create", "bem_server_submit", "bem_server_poll", "bem_server_release", "bem_server_stats_get",
    "bem_server_destroy",
    "bem_cluster_tree_create", "bem_cluster_tree_info", "bem_cluster_tree_query", "bem_cluster_tree_destroy",
]


class BemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class OpOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("m_q", ctypes.c_int32), ("n_theta", ctypes.c_int32),
                ("store_fp32", ctypes.c_int32), ("matrix_free", ctypes.c_int32), ("trial_space", ctypes.c_int32)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int32), ("maxit", ctypes.c_int32),
                ("inner_dtype", ctypes.c_int32), ("max_refine", ctypes.c_int32)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("refinements", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("rel_residual", ctypes.c_double), ("solve_ms", ctypes.c_double)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_int64), ("max_slots", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("inner_dtype", ctypes.c_int32), ("restart", ctypes.c_int32), ("maxit", ctypes.c_int32),
                ("max_refine", ctypes.c_int32), ("tol", ctypes.c_double), ("cache_operators", ctypes.c_int32),
                ("reserved0", ctypes.c_int32)]


class Job(ctypes.Structure):
    _fields_ = [("n_sv", ctypes.c_int64), ("sv_xyz", ctypes.POINTER(ctypes.c_double)),
                ("n_stv", ctypes.c_int64), ("stv_sv", ctypes.POINTER(ctypes.c_int32)),
                ("stv_t", ctypes.POINTER(ctypes.c_double)), ("n_tet", ctypes.c_int64),
                ("tets", ctypes.POINTER(ctypes.c_int32)), ("data_kind", ctypes.c_int32), ("nrhs", ctypes.c_int32),
                ("params", ctypes.POINTER(ctypes.c_double))]


class Completion(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32), ("nrhs", ctypes.c_int32),
                ("n_tet", ctypes.c_int64), ("w", ctypes.POINTER(ctypes.c_double)),
                ("iterations", ctypes.c_int32), ("refinements", ctypes.c_int32), ("rel_residual", ctypes.c_double),
                ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double), ("reserved_bytes", ctypes.c_int64),
                ("cache_hit", ctypes.c_int32), ("reserved0", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("running", ctypes.c_int64), ("peak_running", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("peak_reserved_bytes", ctypes.c_int64),
                ("solves_per_s", ctypes.c_double), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double), ("cache_hits", ctypes.c_int64),
                ("cached_operators", ctypes.c_int64), ("cached_bytes", ctypes.c_int64)]


_lib = None
VP = ctypes.c_void_p
D = ctypes.POINTER(ctypes.c_double)
I32 = ctypes.POINTER(ctypes.c_int32)
I64 = ctypes.POINTER(ctypes.c_int64)


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
        _build.build()
    L = ctypes.CDLL(path)
    L.bem_last_error.restype = ctypes.c_char_p
    L.bem_version.restype = ctypes.c_char_p
    L.bem_context_create.argtypes = [ctypes.c_int, ctypes.POINTER(VP)]
    L.bem_context_destroy.argtypes = [VP]
    L.bem_alu_peaks.argtypes = [VP, D, D]
    L.bem_context_set_tuning.argtypes = [VP, ctypes.c_int, ctypes.c_char_p]
    L.bem_selftest_bounded_wait.argtypes = [VP, D]
    L.bem_cluster_tree_create.argtypes = [ctypes.c_int64, D, ctypes.c_int64, I32, ctypes.c_int32, ctypes.POINTER(VP)]
    L.bem_cluster_tree_info.argtypes = [VP, I64, I64, I32]
    L.bem_cluster_tree_query.argtypes = [VP, D, ctypes.c_int64, I32, I64, I64]
    L.bem_cluster_tree_destroy.argtypes = [VP]
    L.bem_cluster_tree_destroy.restype = None
    L.bem_operator_tuning.argtypes = [VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int), D]
    L.bem_context_destroy.restype = None
    L.bem_mesh_create.argtypes = [VP, ctypes.c_int64, D, ctypes.c_int64, I32, D, ctypes.c_int64, I32,
                                  ctypes.POINTER(VP)]
    L.bem_mesh_create_prisms.argtypes = [VP, ctypes.c_int64, D, ctypes.c_int64, I32, ctypes.c_int32, D,
                                         ctypes.POINTER(VP)]
    L.bem_mesh_info.argtypes = [VP, I64, I64, I64]
    L.bem_mesh_destroy.argtypes = [VP]
    L.bem_mesh_destroy.restype = None
    L.bem_operator_create.argtypes = [VP, VP, ctypes.POINTER(OpOpts), ctypes.POINTER(VP)]
    L.bem_operator_stats.argtypes = [VP, I64, I64, I64, D]
    L.bem_operator_reassemble.argtypes = [VP, VP]
    L.bem_operator_timings.argtypes = [VP, D]
    L.bem_operator_check.argtypes = [VP, I64, D]
    L.bem_operator_work.argtypes = [VP, I64]
    L.bem_operator_export_pattern.argtypes = [VP, I64, I32]
    L.bem_operator_export_dense.argtypes = [VP, D]
    L.bem_operator_pattern_rows.argtypes = [VP, ctypes.c_int64, I32, ctypes.c_int64, I64, I32]
    L.bem_operator_entries.argtypes = [VP, ctypes.c_int64, I32, D]
    L.bem_operator_destroy.argtypes = [VP]
    L.bem_operator_destroy.restype = None
    L.bem_rhs.argtypes = [VP, ctypes.c_int32, ctypes.c_int32, D, D]
    L.bem_rhs_points.argtypes = [VP, ctypes.c_int32, ctypes.c_int32, I64, D, D]
    L.bem_rhs_from_samples.argtypes = [VP, ctypes.c_int32, ctypes.c_int32, D, ctypes.c_int32, D]
    L.bem_matvec.argtypes = [VP, VP, VP, ctypes.c_int32, VP]
    L.bem_matvec_dtype.argtypes = [VP, VP, VP, ctypes.c_int32, ctypes.c_int32, VP]
    L.bem_matvec_noalloc.argtypes = [VP, VP, VP, ctypes.c_int32, VP]
    L.bem_solve.argtypes = [VP, D, D, ctypes.c_int32, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo)]
    L.bem_solve_refined.argtypes = [VP, VP, D, D, ctypes.c_int32, ctypes.POINTER(SolveOpts),
                                    ctypes.POINTER(SolveInfo)]
    L.bem_solve_device.argtypes = [VP, VP, VP, ctypes.c_int32, ctypes.POINTER(SolveOpts),
                                   ctypes.POINTER(SolveInfo), VP]
    L.bem_solve_async.argtypes = [VP, VP, VP, ctypes.c_int32, ctypes.POINTER(SolveOpts), VP, ctypes.POINTER(VP)]
    L.bem_request_wait.argtypes = [VP, ctypes.c_int64, ctypes.POINTER(SolveInfo)]
    L.bem_request_cancel.argtypes = [VP]
    L.bem_request_destroy.argtypes = [VP]
    L.bem_request_destroy.restype = None
    L.bem_inner_potentials.argtypes = [VP, ctypes.c_int64, D, D, I32, ctypes.c_int32, ctypes.c_int32, D]
    L.bem_batch_create.argtypes = [VP, ctypes.c_int32, ctypes.POINTER(VP), ctypes.POINTER(OpOpts), ctypes.POINTER(VP)]
    L.bem_batch_stats.argtypes = [VP, ctypes.POINTER(ctypes.c_int32), I64, I64, D]
    L.bem_batch_solve.argtypes = [VP, ctypes.c_int32, I32, D, ctypes.POINTER(SolveOpts), D, ctypes.POINTER(SolveInfo)]
    L.bem_batch_destroy.argtypes = [VP]
    L.bem_batch_destroy.restype = None
    L.bem_server_create.argtypes = [VP, ctypes.POINTER(ServerOpts), ctypes.POINTER(VP)]
    L.bem_server_submit.argtypes = [VP, ctypes.POINTER(Job), ctypes.POINTER(ctypes.c_uint64)]
    L.bem_server_poll.argtypes = [VP, ctypes.POINTER(Completion), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                  ctypes.c_int64]
    L.bem_server_release.argtypes = [VP, ctypes.c_uint64]
    L.bem_server_stats_get.argtypes = [VP, ctypes.POINTER(ServerStats)]
    L.bem_server_destroy.argtypes = [VP]
    L.bem_server_destroy.restype = None
    for name in EXPORTS:
        if name not in ("bem_context_destroy", "bem_mesh_destroy", "bem_operator_destroy", "bem_last_error",
                        "bem_version", "bem_server_destroy", "bem_batch_destroy", "bem_request_destroy",
                        "bem_cluster_tree_destroy"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def check(status, allow=()):
    if status != BEM_OK and status not in allow:
        raise BemError(status, load().bem_last_error().decode())
    return status


def dptr(a: np.ndarray):
    return a.ctypes.data_as(D)


def iptr(a: np.ndarray):
    return a.ctypes.data_as(I32)


def lptr(a: np.ndarray):
    return a.ctypes.data_as(I64)
