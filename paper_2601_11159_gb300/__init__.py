"""Resistance distance by Lanczos iteration on one GB300 (sm_103a).

Thin Python binding over librd.so (C ABI in include/rd.h). Every step of the
computation runs in the library's CUDA kernels; this module only marshals
arguments: numpy arrays are passed as host pointers, torch CUDA tensors as device
pointers, and the current torch CUDA stream as the stream. Results come back as
torch CUDA tensors when the pair ids are CUDA tensors, else as numpy arrays.

Names follow the C ABI: ``graph_create``, ``graph_set_weights``,
``graph_destroy``, ``query``, ``edge_grad``, ``potential``, ``last_call_stats``,
``status_string``; ``Graph`` bundles them, and ``ResistanceDistance`` is the
``torch.autograd.Function`` whose backward calls ``edge_grad``.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import _lib
from ._lib import (  # noqa: F401
    RD_OK, RD_WARN_NOT_CONVERGED, RD_ERR_INVALID_ARG, RD_ERR_ZERO_DEGREE, RD_ERR_DISCONNECTED,
    RD_ERR_CUDA, RD_ERR_OOM, RD_ERR_TIMEOUT, RD_ERR_NUMERIC, RD_ERR_UNSUPPORTED,
    RD_MODE_FP64, RD_MODE_FP32V_FP64S, RD_MODE_DF64, RD_INPUT_ON_DEVICE, RD_CHECK_SYMMETRY, RD_LABEL_COMPONENTS,
    RD_Q_FIXED_K, RD_Q_NO_DEFLATE, RD_Q_PLAIN, RD_Q_PROFILE, RD_Q_NO_COMPACT, RD_Q_NO_ONCHIP, RD_Q_NO_TUNE,
    RD_Q_NO_GRAPH, RD_Q_EST_DELAYED, RD_Q_DENSE_FIRST, RD_Q_REPLAY_POTENTIAL, RD_Q_NO_CLUSTER,
    RD_Q_NO_DEVICE_LOOP,
)

__all__ = ["Graph", "RDError", "query", "edge_grad", "potential", "graph_create", "graph_destroy",
           "graph_set_weights", "last_call_stats", "status_string", "ResistanceDistance", "lib",
           "query_noalloc", "flow", "power_method"]


def lib():
    return _lib.load()


class RDError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = lib()
        msg = L.rd_status_string(status).decode()
        detail = L.rd_last_error().decode()
        super().__init__(f"{where}: {msg} ({status})" + (f": {detail}" if detail else ""))
        self.status = status


def status_string(status: int) -> str:
    return lib().rd_status_string(int(status)).decode()


def _torch():
    import torch

    return torch


def _is_torch(x) -> bool:
    try:
        import torch

        return isinstance(x, torch.Tensor)
    except ImportError:  # pragma: no cover
        return False


def _stream_ptr(stream=None) -> int:
    if stream is not None:
        return int(stream)
    try:
        import torch

        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except ImportError:  # pragma: no cover
        pass
    return 0


def _arr(x, dtype):
    """(pointer, keep-alive object) for a numpy array or a torch tensor of the given dtype."""
    if x is None:
        return None, None
    if _is_torch(x):
        torch = _torch()
        tdt = {np.int64: torch.int64, np.int32: torch.int32, np.float32: torch.float32,
               np.float64: torch.float64}[dtype]
        if x.dtype != tdt or not x.is_contiguous():
            x = x.to(tdt).contiguous()
        if x.device.type == "cpu" and x.numel() > 0:
            return x.data_ptr(), x
        return (x.data_ptr() if x.numel() > 0 else None), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return (a.ctypes.data if a.size > 0 else None), a


def _check(st: int, where: str, ok=(RD_OK, RD_WARN_NOT_CONVERGED)):
    if st not in ok:
        raise RDError(st, where)
    return st


def _opts(k_max=1000, rel_tol=1e-7, resid_tol=0.0, mode="fp32", rhs_tile=0, rows_per_warp=0, chunk_steps=0,
          fixed_k=False, deflate=True, plain=False, profile=False, kernel=0, compact=True,
          onchip=True, tune=True, graph=True, estimate="geometric", sparse_first=True,
          potential_mode="direct", cluster=True, device_loop=True) -> _lib.QueryOpts:
    """rd_query_opts from keywords (each documented in include/rd.h): k_max, rel_tol,
    resid_tol, mode ("fp32" FP32 vectors with FP64 scalars, "fp64", "df64"), rhs_tile,
    rows_per_warp, chunk_steps, kernel ("tuned", "group", "stream", "group_sorted", "tasks",
    "async" or its number); the booleans clear or set one flag each: fixed_k (RD_Q_FIXED_K),
    deflate (RD_Q_NO_DEFLATE), plain (RD_Q_PLAIN), profile (RD_Q_PROFILE), compact
    (RD_Q_NO_COMPACT), onchip (RD_Q_NO_ONCHIP), tune (RD_Q_NO_TUNE), graph (RD_Q_NO_GRAPH),
    sparse_first (RD_Q_DENSE_FIRST), cluster (RD_Q_NO_CLUSTER), device_loop
    (RD_Q_NO_DEVICE_LOOP); estimate "geometric" or "delayed" (RD_Q_EST_DELAYED);
    potential_mode "direct" or "replay" (RD_Q_REPLAY_POTENTIAL)."""
    o = _lib.QueryOpts()
    lib().rd_query_opts_init(C.byref(o))
    o.k_max = int(k_max)
    o.rel_tol = float(rel_tol)
    o.resid_tol = float(resid_tol)
    if mode in ("fp64", RD_MODE_FP64):
        o.mode = RD_MODE_FP64
    elif mode in ("fp32", RD_MODE_FP32V_FP64S):
        o.mode = RD_MODE_FP32V_FP64S
    elif mode in ("df64", RD_MODE_DF64):
        o.mode = RD_MODE_DF64
    else:
        raise ValueError(f"unknown mode {mode!r}")
    o.rhs_tile = int(rhs_tile)
    o.rows_per_warp = int(rows_per_warp)
    o.chunk_steps = int(chunk_steps)
    o.kernel = ({"tuned": 0, "group": 1, "stream": 2, "group_sorted": 3, "tasks": 4, "async": 5}.get(kernel, kernel)
                if isinstance(kernel, str) else int(kernel))
    o.flags = ((RD_Q_FIXED_K if fixed_k else 0) | (0 if deflate else RD_Q_NO_DEFLATE) |
               (RD_Q_PLAIN if plain else 0) | (RD_Q_PROFILE if profile else 0) |
               (0 if compact else RD_Q_NO_COMPACT) | (0 if onchip else RD_Q_NO_ONCHIP) |
               (0 if tune else RD_Q_NO_TUNE) | (0 if graph else RD_Q_NO_GRAPH) |
               (RD_Q_EST_DELAYED if estimate == "delayed" else 0) | (0 if sparse_first else RD_Q_DENSE_FIRST) |
               (RD_Q_REPLAY_POTENTIAL if potential_mode == "replay" else 0) | (0 if cluster else RD_Q_NO_CLUSTER) |
               (0 if device_loop else RD_Q_NO_DEVICE_LOOP))
    if estimate not in ("geometric", "delayed"):
        raise ValueError(f"unknown estimate {estimate!r}")
    if potential_mode not in ("direct", "replay"):
        raise ValueError(f"unknown potential_mode {potential_mode!r}")
    return o


def _out(like_device: bool, n: int, dtype):
    if like_device:
        torch = _torch()
        tdt = {np.float64: torch.float64, np.int32: torch.int32, np.float32: torch.float32}[dtype]
        t = torch.empty(n, dtype=tdt, device="cuda")
        return t, (t.data_ptr() if n > 0 else None)
    a = np.empty(n, dtype=dtype)
    return a, (a.ctypes.data if n > 0 else None)


# ------------------------------------------------------------------ C names
def graph_create(row_ptr, col, w=None, flags: int = RD_LABEL_COMPONENTS, stream=None) -> int:
    """rd_graph_create: returns an opaque handle (int)."""
    rp, k1 = _arr(row_ptr, np.int64)
    cp, k2 = _arr(col, np.int32)
    wp, k3 = _arr(w, np.float32)
    n = (k1.numel() if _is_torch(k1) else k1.size) - 1
    nnz = k2.numel() if _is_torch(k2) else k2.size
    h = C.c_void_p()
    st = lib().rd_graph_create(C.byref(h), n, nnz, rp, cp, wp, flags, _stream_ptr(stream))
    _check(st, "rd_graph_create", ok=(RD_OK,))
    return h.value


def graph_set_weights(handle: int, w, stream=None):
    wp, keep = _arr(w, np.float32)
    _check(lib().rd_graph_set_weights(handle, wp, _stream_ptr(stream)), "rd_graph_set_weights", ok=(RD_OK,))


def graph_destroy(handle: int):
    if handle:
        lib().rd_graph_destroy(handle)


def last_call_stats(handle: int) -> dict:
    s = _lib.CallStats()
    _check(lib().rd_last_call_stats(handle, C.byref(s)), "rd_last_call_stats", ok=(RD_OK,))
    return {f: getattr(s, f) for f, _ in _lib.CallStats._fields_}


@dataclass
class QueryResult:
    r: object
    iters: object
    err: object
    status: object
    call_status: int


def query(handle: int, s, t, stream=None, **kw) -> QueryResult:
    """rd_query over pairs (s[i], t[i]); keyword options as in ``_opts``."""
    dev = _is_torch(s) and s.is_cuda
    sp, ks = _arr(s, np.int32)
    tp_, kt = _arr(t, np.int32)
    P = ks.numel() if _is_torch(ks) else ks.size
    r, rp = _out(dev, P, np.float64)
    it, ip = _out(dev, P, np.int32)
    er, ep = _out(dev, P, np.float64)
    ps, pp = _out(dev, P, np.int32)
    o = _opts(**kw)
    st = lib().rd_query(handle, sp, tp_, P, C.byref(o), rp, ip, ep, pp, _stream_ptr(stream))
    _check(st, "rd_query")
    return QueryResult(r, it, er, ps, st)


def edge_grad(handle: int, nnz_in: int, s, t, grad_r=None, stream=None, want_r: bool = True, **kw):
    """rd_edge_grad: returns (grad_w[nnz], r[P])."""
    dev = _is_torch(s) and s.is_cuda
    sp, ks = _arr(s, np.int32)
    tp_, kt = _arr(t, np.int32)
    gp, kg = _arr(grad_r, np.float64)
    P = ks.numel() if _is_torch(ks) else ks.size
    gw, gwp = _out(dev, nnz_in, np.float32)
    r, rp = _out(dev, P, np.float64) if want_r else (None, None)
    o = _opts(**kw)
    st = lib().rd_edge_grad(handle, sp, tp_, P, gp, C.byref(o), gwp, rp, _stream_ptr(stream))
    _check(st, "rd_edge_grad")
    return gw, r


def potential(handle: int, n: int, s, t, stream=None, **kw):
    """rd_potential: returns (phi[P, n] float32, r[P])."""
    dev = _is_torch(s) and s.is_cuda
    sp, ks = _arr(s, np.int32)
    tp_, kt = _arr(t, np.int32)
    P = ks.numel() if _is_torch(ks) else ks.size
    phi, php = _out(dev, P * n, np.float32)
    r, rp = _out(dev, P, np.float64)
    o = _opts(**kw)
    st = lib().rd_potential(handle, sp, tp_, P, C.byref(o), php, rp, _stream_ptr(stream))
    _check(st, "rd_potential")
    return phi.reshape(P, n), r


def flow(handle: int, nnz_in: int, s, t, stream=None, **kw):
    """rd_flow: returns (f[P, nnz] float32 potential differences per stored entry, r[P])."""
    dev = _is_torch(s) and s.is_cuda
    sp, ks = _arr(s, np.int32)
    tp_, kt = _arr(t, np.int32)
    P = ks.numel() if _is_torch(ks) else ks.size
    f, fp = _out(dev, P * nnz_in, np.float32)
    r, rp = _out(dev, P, np.float64)
    o = _opts(**kw)
    st = lib().rd_flow(handle, sp, tp_, P, C.byref(o), fp, rp, _stream_ptr(stream))
    _check(st, "rd_flow")
    return f.reshape(P, nnz_in), r


def power_method(handle: int, s, t, steps: int, mode: str = "fp64", history: bool = False, stream=None):
    """rd_power_method (Algorithm 1): returns (rbar[P], hist[steps+1, P] or None)."""
    dev = _is_torch(s) and s.is_cuda
    sp, ks = _arr(s, np.int32)
    tp_, kt = _arr(t, np.int32)
    P = ks.numel() if _is_torch(ks) else ks.size
    r, rp = _out(dev, P, np.float64)
    hist, hp = _out(dev, P * (steps + 1), np.float64) if history else (None, None)
    m = RD_MODE_FP64 if mode in ("fp64", RD_MODE_FP64) else RD_MODE_FP32V_FP64S
    st = lib().rd_power_method(handle, sp, tp_, P, int(steps), m, rp, hp, _stream_ptr(stream))
    _check(st, "rd_power_method", ok=(RD_OK,))
    return r, (None if hist is None else hist.reshape(steps + 1, P))


def _noalloc_tensor(x, name: str, dtype, min_numel: int = 0):
    """Pointer of a tensor handed to rd_query_noalloc as is: a contiguous CUDA tensor of the
    exact dtype on the current device. Nothing is converted, because a conversion would
    allocate device memory, which is what this entry point's callers cannot do."""
    torch = _torch()
    if not (_is_torch(x) and x.is_cuda):
        raise TypeError(f"query_noalloc: {name} must be a CUDA tensor")
    if x.device.index != torch.cuda.current_device():
        raise ValueError(f"query_noalloc: {name} is on {x.device}, not on the current device")
    if x.dtype != dtype:
        raise TypeError(f"query_noalloc: {name} must be {dtype}, got {x.dtype}")
    if not x.is_contiguous():
        raise TypeError(f"query_noalloc: {name} must be contiguous")
    if x.numel() < min_numel:
        raise ValueError(f"query_noalloc: {name} holds {x.numel()} elements, needs at least {min_numel}")
    return x.data_ptr() if x.numel() > 0 else None


def query_noalloc(row_ptr, col, w, s, t, stream=None, **kw):
    """rd_query_noalloc for callers that cannot allocate device memory: every array must be a
    contiguous CUDA tensor of the C ABI's type on the current device (row_ptr int64, col int32,
    w float32 or None, s and t int32 of equal length); nothing is converted. The graph is used
    in place and no handle is created. Returns (r, iters) as CUDA tensors; pass
    ``out=(r, iters)`` (float64 and int32, at least len(s) elements each) to reuse
    preallocated outputs, so that the call itself allocates nothing."""
    torch = _torch()
    out = kw.pop("out", None)
    rp = _noalloc_tensor(row_ptr, "row_ptr", torch.int64, 1)
    cp = _noalloc_tensor(col, "col", torch.int32)
    wp = None if w is None else _noalloc_tensor(w, "w", torch.float32, col.numel())
    sp = _noalloc_tensor(s, "s", torch.int32)
    P = s.numel()
    tp_ = _noalloc_tensor(t, "t", torch.int32)
    if t.numel() != P:
        raise ValueError(f"query_noalloc: s and t differ in length ({P} and {t.numel()})")
    if out is None:
        r, rp_ = _out(True, P, np.float64)
        it, ip = _out(True, P, np.int32)
    else:
        r, it = out
        rp_ = _noalloc_tensor(r, "out[0] (r)", torch.float64, P)
        ip = _noalloc_tensor(it, "out[1] (iters)", torch.int32, P)
    n = row_ptr.numel() - 1
    o = _opts(**kw)
    st = lib().rd_query_noalloc(n, col.numel(), rp, cp, wp, sp, tp_, P, C.byref(o), rp_, ip, _stream_ptr(stream))
    _check(st, "rd_query_noalloc")
    return r, it


# -------------------------------------------------------------------- Graph
class Graph:
    """A device-resident graph (symmetric CSR, optional positive edge weights)."""

    def __init__(self, row_ptr, col, w=None, check_symmetry: bool = False, label_components: bool = True,
                 stream=None):
        flags = (RD_CHECK_SYMMETRY if check_symmetry else 0) | (RD_LABEL_COMPONENTS if label_components else 0)
        self.handle = graph_create(row_ptr, col, w, flags, stream)
        n, nnz, wt, nc = C.c_int64(), C.c_int64(), C.c_int32(), C.c_int32()
        lib().rd_graph_info(self.handle, C.byref(n), C.byref(nnz), C.byref(wt), C.byref(nc))
        self.n, self.nnz, self.weighted, self.ncomponents = n.value, nnz.value, bool(wt.value), nc.value
        self.nnz_in = len(col)

    @classmethod
    def from_csr(cls, g, **kw) -> "Graph":
        """From any object with ``row_ptr``, ``col`` and ``w`` attributes."""
        return cls(g.row_ptr, g.col, g.w, **kw)

    def set_weights(self, w, stream=None):
        graph_set_weights(self.handle, w, stream)
        self.weighted = True

    def query(self, s, t, **kw) -> QueryResult:
        return query(self.handle, s, t, **kw)

    def edge_grad(self, s, t, grad_r=None, **kw):
        return edge_grad(self.handle, self.nnz_in, s, t, grad_r, **kw)

    def potential(self, s, t, **kw):
        return potential(self.handle, self.n, s, t, **kw)

    def flow(self, s, t, **kw):
        return flow(self.handle, self.nnz_in, s, t, **kw)

    def triangle_weights(self, device: bool = False):
        """rd_triangle_weights: float32[nnz] triangle counts per stored entry (1 where none)."""
        w, wp = _out(device, self.nnz, np.float32)
        _check(lib().rd_triangle_weights(self.handle, wp, _stream_ptr(None)), "rd_triangle_weights", ok=(RD_OK,))
        return w

    def power_method(self, s, t, steps: int, **kw):
        return power_method(self.handle, s, t, steps, **kw)

    def last_stats(self) -> dict:
        return last_call_stats(self.handle)

    def autotune(self, npairs: int, stream=None, **kw) -> dict:
        """rd_autotune: time the SpMM candidates for npairs pairs and keep the fastest on this
        graph; returns the configuration a query of npairs pairs now uses."""
        tile, rpw, kern = C.c_int32(), C.c_int32(), C.c_int32()
        o = _opts(**kw)
        _check(lib().rd_autotune(self.handle, int(npairs), C.byref(o), C.byref(tile), C.byref(rpw), C.byref(kern),
                                 _stream_ptr(stream)), "rd_autotune", ok=(RD_OK,))
        return {"rhs_tile": tile.value, "rows_per_warp": rpw.value, "kernel": kern.value}

    def close(self):
        graph_destroy(getattr(self, "handle", None))
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _make_autograd():
    torch = _torch()

    class ResistanceDistance(torch.autograd.Function):
        """r = ResistanceDistance.apply(w, graph, s, t, opts): resistance distances of the pairs under
        edge weights ``w`` (float32 CUDA tensor, one per stored CSR entry, kept symmetric). The
        backward pass calls rd_edge_grad, which recomputes the forward recurrence and builds the
        potentials during those steps from the LDL^T factors of I - T_i (the direct update; no
        basis is stored and no second pass runs unless opts asks for potential_mode="replay")."""

        @staticmethod
        def forward(ctx, w, graph, s, t, opts=None):
            opts = dict(opts or {})
            graph.set_weights(w.detach())
            res = graph.query(s, t, **opts)
            ctx.graph, ctx.s, ctx.t, ctx.opts = graph, s, t, opts
            ctx.save_for_backward(w)
            return res.r

        @staticmethod
        def backward(ctx, grad_r):
            (w,) = ctx.saved_tensors
            ctx.graph.set_weights(w.detach())
            gw, _ = ctx.graph.edge_grad(ctx.s, ctx.t, grad_r.detach().to(torch.float64).contiguous(),
                                        want_r=False, **ctx.opts)
            return gw.to(w.dtype), None, None, None, None

    return ResistanceDistance


def __getattr__(name):
    if name == "ResistanceDistance":
        cls = _make_autograd()
        globals()["ResistanceDistance"] = cls
        return cls
    raise AttributeError(name)
