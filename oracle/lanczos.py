"""Oracle, Lanczos part: Python access to the plain C FP64 Lanczos of ``lanczos_ref.c``
(Section 3, Algorithm 3; potential from Section 6.3, Algorithm 5).

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the benchmark's
CPU baseline; never by the product library. It is compiled with gcc on first use
(``build()``) into ``oracle/_build/liboracle.so``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lanczos_ref.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


_SO_TIMING = os.path.join(_BUILD, "liboracle_O3.so")
_lib_timing = None


def build(force: bool = False, src: str = _SRC, out: str = _SO, opt: str = "-O2") -> str:
    """Compile the C oracle (plain -O2, OpenMP over pairs; no machine-specific flags)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", opt, "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, out)
    return out


def build_timing(force: bool = False) -> str:
    """The same source compiled with -O3 for the timed CPU baseline (the pinned build used by
    the tests stays -O2). No -march=native: host code here must build and give the same
    results on the x86 and Arm hosts, and -O3 alone already vectorises for the baseline ISA
    of each."""
    return build(force, _SRC, _SO_TIMING, "-O3")


def load_timing():
    """The -O3 build of the oracle (see build_timing), for timing only."""
    global _lib_timing
    if _lib_timing is None:
        lib = load(build_timing())  # load() takes the module lock itself
        with _lock:
            if _lib_timing is None:
                _lib_timing = lib
    return _lib_timing


def load(path: str = None):
    """Load (building if needed) the oracle library and declare its signatures."""
    global _lib
    with _lock:
        if path is None and _lib is not None:
            return _lib
        so = path or build()
        lib = C.CDLL(so)
        P = C.c_void_p
        lib.orc_degrees.argtypes = [C.c_int64, P, P, P]
        lib.orc_degrees.restype = None
        lib.orc_lanczos_pair.argtypes = [C.c_int64, P, P, P, P, C.c_int32, C.c_int32, C.c_int, C.c_double,
                                         P, P, P, P, P, P]
        lib.orc_lanczos_pair.restype = C.c_int
        lib.orc_lanczos_batch.argtypes = [C.c_int64, P, P, P, P, P, C.c_int64, C.c_int, C.c_double, C.c_int, P, P]
        lib.orc_lanczos_batch.restype = C.c_int
        lib.orc_num_threads.argtypes = []
        lib.orc_num_threads.restype = C.c_int
        if path is None:
            _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    w = None if g.w is None else np.ascontiguousarray(g.w, dtype=np.float32)
    return rp, col, w


def degrees(g, lib=None) -> np.ndarray:
    lib = lib or load()
    rp, col, w = _csr(g)
    d = np.empty(g.n, dtype=np.float64)
    lib.orc_degrees(g.n, _ptr(rp), _ptr(w), _ptr(d))
    return d


def lanczos_pair(g, s: int, t: int, k_max: int, stop_tol: float = 0.0, want_basis: bool = False,
                 want_potential: bool = False, lib=None) -> dict:
    """Run Algorithm 3 for one pair; returns r, k, r_hist, alpha, beta (and V, phi on request)."""
    lib = lib or load()
    rp, col, w = _csr(g)
    deg = degrees(g, lib)
    r = np.zeros(1)
    r_hist = np.zeros(k_max)
    alpha = np.zeros(k_max)
    beta = np.zeros(k_max + 1)
    V = np.zeros((k_max + 1, g.n)) if (want_basis or want_potential) else None
    phi = np.zeros(g.n) if want_potential else None
    k = lib.orc_lanczos_pair(g.n, _ptr(rp), _ptr(col), _ptr(w), _ptr(deg), int(s), int(t), int(k_max),
                             float(stop_tol), _ptr(r), _ptr(r_hist), _ptr(alpha), _ptr(beta), _ptr(V), _ptr(phi))
    out = dict(r=float(r[0]), k=int(k), r_hist=r_hist[:k], alpha=alpha[:k], beta=beta[:k + 1])
    if V is not None:
        out["V"] = V[:k + 1].T.copy()  # n x (k+1): columns v_1 .. v_{k+1}
    if phi is not None:
        out["phi"] = phi
    return out


def lanczos_batch(g, s, t, k_max: int, stop_tol: float = 0.0, threads: int = 0, lib=None):
    """Many pairs (one per OpenMP thread). Returns (r[P], k[P], threads_used)."""
    lib = lib or load()
    rp, col, w = _csr(g)
    s = np.ascontiguousarray(s, dtype=np.int32)
    t = np.ascontiguousarray(t, dtype=np.int32)
    r = np.zeros(s.size)
    k = np.zeros(s.size, dtype=np.int32)
    used = lib.orc_lanczos_batch(g.n, _ptr(rp), _ptr(col), _ptr(w), _ptr(s), _ptr(t), s.size, int(k_max),
                                 float(stop_tol), int(threads), _ptr(r), _ptr(k))
    return r, k, used


def num_threads(lib=None) -> int:
    return (lib or load()).orc_num_threads()
