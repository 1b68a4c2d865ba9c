"""Oracle, dense part: resistance distance, potentials and edge-weight gradients from
the Laplacian pseudo-inverse, in FP64, for small graphs (n up to a few thousand).

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the benchmark's
CPU baseline; never by the product library.

* Section 2.1, Definition of RD: r(s,t) = (e_s - e_t)^T L^+ (e_s - e_t), L = D - W
  (weights as in "directly generalized to weighted graphs").
* L^+ for a connected graph: L + J/n is invertible (J = all-ones), and
  L^+ = (L + J/n)^{-1} - J/n, because L and J/n share the eigenbasis, L's null
  vector 1/sqrt(n) gets eigenvalue 1 in L + J/n, and all other eigenvectors are
  orthogonal to 1.
* Section 6.3, Definition electric_flow: phi = L^+ (e_s - e_t), f(e) = phi(u) - phi(v).
* Edge-weight derivative (not in the paper; standard matrix calculus): with
  L = sum_e w_e b_e b_e^T, d L^+ / d w_e = -L^+ b_e b_e^T L^+ on the range of L, so
  d r / d w_e = -(phi(u) - phi(v))^2. Each undirected edge is stored twice in the
  CSR; each stored copy receives half of the edge derivative.
"""
from __future__ import annotations

import numpy as np


def laplacian(n, row_ptr, col, w=None) -> np.ndarray:
    """Dense L = D - W from symmetric CSR (weights FP32 promoted to FP64)."""
    L = np.zeros((n, n), dtype=np.float64)
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    vals = np.ones(len(col), dtype=np.float64) if w is None else np.asarray(w, dtype=np.float64)
    np.add.at(L, (rows, np.asarray(col, dtype=np.int64)), -vals)
    L[np.diag_indices(n)] -= L.sum(axis=1)
    return L


def pinv_laplacian(L: np.ndarray) -> np.ndarray:
    """L^+ = (L + J/n)^{-1} - J/n (connected graph)."""
    n = L.shape[0]
    J = np.full((n, n), 1.0 / n)
    return np.linalg.inv(L + J) - J


class DenseRD:
    """Resistance distances of one small graph from its dense pseudo-inverse."""

    def __init__(self, n, row_ptr, col, w=None):
        self.n = n
        self.row_ptr = np.asarray(row_ptr, dtype=np.int64)
        self.col = np.asarray(col, dtype=np.int64)
        self.w = None if w is None else np.asarray(w, dtype=np.float64)
        self.L = laplacian(n, row_ptr, col, w)
        self.Lp = pinv_laplacian(self.L)

    @classmethod
    def of(cls, g):
        return cls(g.n, g.row_ptr, g.col, g.w)

    def r(self, s, t) -> np.ndarray:
        """r(s,t) for arrays of pairs (0 where s == t)."""
        s = np.atleast_1d(np.asarray(s, dtype=np.int64))
        t = np.atleast_1d(np.asarray(t, dtype=np.int64))
        Lp = self.Lp
        return Lp[s, s] + Lp[t, t] - 2.0 * Lp[s, t]

    def potential(self, s: int, t: int) -> np.ndarray:
        """phi = L^+ (e_s - e_t)."""
        return self.Lp[:, s] - self.Lp[:, t]

    def edge_grad(self, s, t, gbar=None) -> np.ndarray:
        """Per stored CSR entry e = (u -> v): 0.5 * sum_p gbar_p * d r_p / d w_uv
        = -0.5 * sum_p gbar_p (phi_p(u) - phi_p(v))^2 (gbar = ones when None)."""
        s = np.atleast_1d(np.asarray(s, dtype=np.int64))
        t = np.atleast_1d(np.asarray(t, dtype=np.int64))
        gbar = np.ones(s.size) if gbar is None else np.asarray(gbar, dtype=np.float64)
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        out = np.zeros(len(self.col), dtype=np.float64)
        for p in range(s.size):
            phi = self.potential(int(s[p]), int(t[p]))
            out -= 0.5 * gbar[p] * (phi[rows] - phi[self.col]) ** 2
        return out
