"""Closed forms and brute-force references used to pin the oracle (test-only).

Nothing here calls the oracle or the CUDA library; each value follows from
circuit theory or an exact spectral decomposition written out independently.
"""
from __future__ import annotations

import numpy as np


def complete_graph_r(n: int) -> float:
    """K_n: every pair has r = 2/n."""
    return 2.0 / n


def cycle_r(n: int, hops: int) -> float:
    """C_n: two arcs of hops and n-hops unit resistors in parallel."""
    return hops * (n - hops) / n


def tree_r(parent: np.ndarray, w_of_child: np.ndarray, s: int, t: int) -> float:
    """Tree: r = sum of 1/w over the unique path (resistors in series).
    parent[0] = 0 is the root; w_of_child[v] is the weight of edge (v, parent[v])."""
    def ancestors(v):
        out = [v]
        while v != 0:
            v = int(parent[v])
            out.append(v)
        return out

    As, At = ancestors(s), ancestors(t)
    common = set(As) & set(At)
    r = 0.0
    for chain in (As, At):
        for v in chain:
            if v in common:
                break
            r += 1.0 / float(w_of_child[v])
    return r


def grid_r(nx: int, ny: int, s: int, t: int) -> float:
    """Unweighted nx-by-ny 4-neighbour grid (vertex id y*nx + x), exact spectral sum.

    L = L_P(nx) (x) I + I (x) L_P(ny); the path Laplacian L_P(N) has eigenpairs
    lambda_i = 2 - 2 cos(pi i / N), phi_i(x) = c_i cos(pi i (x + 1/2) / N) with
    c_0 = sqrt(1/N), c_i = sqrt(2/N). r(s,t) = sum over (i,j) != (0,0) of
    (phi_i(sx) phi_j(sy) - phi_i(tx) phi_j(ty))^2 / (lambda_i + lambda_j)."""
    def basis(N):
        i = np.arange(N)[:, None]
        x = np.arange(N)[None, :]
        c = np.where(i == 0, np.sqrt(1.0 / N), np.sqrt(2.0 / N))
        return c * np.cos(np.pi * i * (x + 0.5) / N), 2.0 - 2.0 * np.cos(np.pi * np.arange(N) / N)

    Bx, lx = basis(nx)
    By, ly = basis(ny)
    sx, sy = s % nx, s // nx
    tx, ty = t % nx, t // nx
    diff = np.outer(Bx[:, sx], By[:, sy]) - np.outer(Bx[:, tx], By[:, ty])
    lam = lx[:, None] + ly[None, :]
    lam[0, 0] = 1.0
    diff[0, 0] = 0.0
    return float(np.sum(diff * diff / lam))


def series(*rs: float) -> float:
    return float(sum(rs))


def parallel(*rs: float) -> float:
    return 1.0 / float(sum(1.0 / r for r in rs))


def normalized_adjacency(n, row_ptr, col, w=None) -> np.ndarray:
    """Dense Ahat = D^{-1/2} W D^{-1/2} built directly from the CSR (for invariant checks)."""
    W = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    vals = np.ones(len(col)) if w is None else np.asarray(w, dtype=np.float64)
    np.add.at(W, (rows, np.asarray(col, dtype=np.int64)), vals)
    d = W.sum(axis=1)
    isd = 1.0 / np.sqrt(d)
    return isd[:, None] * W * isd[None, :]
