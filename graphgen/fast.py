"""ctypes access to graphgen/fastgen.c (R-MAT endpoints and edge list -> symmetric CSR),
compiled with gcc on first use into graphgen/_build/libfastgen.so. Input preparation only."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fastgen.c")
_SO = os.path.join(_HERE, "_build", "libfastgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            lib.gg_rmat_edges.argtypes = [C.c_int, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_uint64,
                                          C.c_uint64, P, P]
            lib.gg_rmat_edges.restype = None
            lib.gg_csr_from_edges.argtypes = [C.c_int64, C.c_int64, P, P, P, P]
            lib.gg_csr_from_edges.restype = C.c_int64
            lib.gg_ba_edges.argtypes = [C.c_int64, C.c_int, C.c_uint64, C.c_uint64, P, P]
            lib.gg_ba_edges.restype = C.c_int64
            _lib = lib
        return _lib


def rmat_edges(scale: int, m: int, a: float, b: float, c: float, seed: int, stream: int):
    lib = load()
    u = np.empty(m, dtype=np.int64)
    v = np.empty(m, dtype=np.int64)
    lib.gg_rmat_edges(scale, m, a, b, c, seed & 0xFFFFFFFFFFFFFFFF, stream, u.ctypes.data, v.ctypes.data)
    return u, v


def csr_from_edges(n: int, u: np.ndarray, v: np.ndarray):
    """(row_ptr int64[n+1], col int32[nnz]) of the symmetric, deduplicated, loop-free graph."""
    lib = load()
    u = np.ascontiguousarray(u, dtype=np.int64)
    v = np.ascontiguousarray(v, dtype=np.int64)
    row_ptr = np.empty(n + 1, dtype=np.int64)
    col = np.empty(2 * u.size, dtype=np.int32)
    nnz = lib.gg_csr_from_edges(n, u.size, u.ctypes.data, v.ctypes.data, row_ptr.ctypes.data, col.ctypes.data)
    return row_ptr, col[:nnz].copy()


def ba_edges(n: int, m_attach: int, seed: int, stream: int):
    lib = load()
    m0 = m_attach + 1
    cap = m0 * (m0 - 1) // 2 + (n - m0) * m_attach + 16
    src = np.empty(cap, dtype=np.int64)
    dst = np.empty(cap, dtype=np.int64)
    k = lib.gg_ba_edges(n, m_attach, seed & 0xFFFFFFFFFFFFFFFF, stream, src.ctypes.data, dst.ctypes.data)
    return src[:k], dst[:k]
