"""ctypes declarations of librd.so (the C ABI in include/rd.h).

Loading fails loudly when the library has not been built: there is no CPU
fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librd.so")

RD_ABI_VERSION = 1

RD_OK = 0
RD_WARN_NOT_CONVERGED = 1
RD_ERR_INVALID_ARG = -1
RD_ERR_ZERO_DEGREE = -2
RD_ERR_DISCONNECTED = -3
RD_ERR_CUDA = -4
RD_ERR_OOM = -5
RD_ERR_TIMEOUT = -6
RD_ERR_NUMERIC = -7
RD_ERR_UNSUPPORTED = -8

RD_MODE_FP64 = 0
RD_MODE_DF64 = 2
RD_MODE_FP32V_FP64S = 1

RD_INPUT_ON_DEVICE = 1
RD_CHECK_SYMMETRY = 2
RD_LABEL_COMPONENTS = 4

RD_Q_FIXED_K = 1
RD_Q_NO_DEFLATE = 2
RD_Q_PLAIN = 4
RD_Q_PROFILE = 8
RD_Q_NO_COMPACT = 16
RD_Q_NO_ONCHIP = 32
RD_Q_NO_TUNE = 64
RD_Q_NO_GRAPH = 128
RD_Q_EST_DELAYED = 256
RD_Q_DENSE_FIRST = 512
RD_Q_REPLAY_POTENTIAL = 1024
RD_Q_NO_CLUSTER = 2048
RD_Q_NO_DEVICE_LOOP = 4096


class QueryOpts(C.Structure):
    _fields_ = [
        ("k_max", C.c_int32),
        ("rel_tol", C.c_double),
        ("resid_tol", C.c_double),
        ("mode", C.c_int32),
        ("rhs_tile", C.c_int32),
        ("rows_per_warp", C.c_int32),
        ("chunk_steps", C.c_int32),
        ("flags", C.c_uint32),
        ("kernel", C.c_int32),
    ]


class CallStats(C.Structure):
    _fields_ = [
        ("launches", C.c_int64),
        ("spmm_launches", C.c_int64),
        ("spmm_ms", C.c_double),
        ("steps", C.c_int32),
        ("rhs_tile", C.c_int32),
        ("rows_per_warp", C.c_int32),
        ("nnz_lanes", C.c_int32),
        ("kernel", C.c_int32),
        ("ld", C.c_int64),
        ("spmm_bytes", C.c_double),
        ("compactions", C.c_int32),
        ("tuned", C.c_int32),
        ("row_order", C.c_int32),
        ("sparse_first", C.c_int32),
        ("onchip_ctas", C.c_int32),
        ("device_loop", C.c_int32),
    ]


EXPORTS = [
    "rd_query_opts_init",
    "rd_graph_create",
    "rd_graph_set_weights",
    "rd_graph_destroy",
    "rd_graph_info",
    "rd_query",
    "rd_edge_grad",
    "rd_potential",
    "rd_flow",
    "rd_power_method",
    "rd_triangle_weights",
    "rd_query_noalloc",
    "rd_autotune",
    "rd_last_call_stats",
    "rd_status_string",
    "rd_last_error",
]

_lib = None


def declare(lib):
    P = C.c_void_p
    lib.rd_query_opts_init.argtypes = [C.POINTER(QueryOpts)]
    lib.rd_query_opts_init.restype = None
    lib.rd_graph_create.argtypes = [C.POINTER(P), C.c_int64, C.c_int64, P, P, P, C.c_uint32, P]
    lib.rd_graph_create.restype = C.c_int
    lib.rd_graph_set_weights.argtypes = [P, P, P]
    lib.rd_graph_set_weights.restype = C.c_int
    lib.rd_graph_destroy.argtypes = [P]
    lib.rd_graph_destroy.restype = C.c_int
    lib.rd_graph_info.argtypes = [P, P, P, P, P]
    lib.rd_graph_info.restype = C.c_int
    lib.rd_query.argtypes = [P, P, P, C.c_int64, C.POINTER(QueryOpts), P, P, P, P, P]
    lib.rd_query.restype = C.c_int
    lib.rd_edge_grad.argtypes = [P, P, P, C.c_int64, P, C.POINTER(QueryOpts), P, P, P]
    lib.rd_edge_grad.restype = C.c_int
    lib.rd_potential.argtypes = [P, P, P, C.c_int64, C.POINTER(QueryOpts), P, P, P]
    lib.rd_potential.restype = C.c_int
    lib.rd_flow.argtypes = [P, P, P, C.c_int64, C.POINTER(QueryOpts), P, P, P]
    lib.rd_flow.restype = C.c_int
    lib.rd_power_method.argtypes = [P, P, P, C.c_int64, C.c_int32, C.c_int32, P, P, P]
    lib.rd_power_method.restype = C.c_int
    lib.rd_triangle_weights.argtypes = [P, P, P]
    lib.rd_triangle_weights.restype = C.c_int
    lib.rd_query_noalloc.argtypes = [C.c_int64, C.c_int64, P, P, P, P, P, C.c_int64, C.POINTER(QueryOpts), P, P, P]
    lib.rd_query_noalloc.restype = C.c_int
    lib.rd_autotune.argtypes = [P, C.c_int64, C.POINTER(QueryOpts), P, P, P, P]
    lib.rd_autotune.restype = C.c_int
    lib.rd_last_call_stats.argtypes = [P, C.POINTER(CallStats)]
    lib.rd_last_call_stats.restype = C.c_int
    lib.rd_status_string.argtypes = [C.c_int]
    lib.rd_status_string.restype = C.c_char_p
    lib.rd_last_error.argtypes = []
    lib.rd_last_error.restype = C.c_char_p
    return lib


def load(path: str = LIB_PATH):
    """Load librd.so; raises if it is missing (run ``python -m paper_2601_11159_gb300.build``)."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"librd.so not built at {path}; build it with paper_2601_11159_gb300.build.build()")
    lib = declare(C.CDLL(path))
    if path == LIB_PATH:
        _lib = lib
    return lib
