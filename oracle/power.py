"""Oracle, Power Method part (Section 2.2, Algorithm 1): the truncated lazy-walk series

    rbar_l = sum_{i=0..l} [ r_i(s)/(2 d_s) - r_i(t)/(2 d_t) ],  r_0 = e_s - e_t,
    r_{i+1} = (I/2 + P/2) r_i,  P = A D^{-1},

in FP64 with scipy sparse products, in the order the algorithm states.

TEST INFRASTRUCTURE ONLY: used by the tests; never by the product library.
"""
from __future__ import annotations

import numpy as np


def power_method(g, s: int, t: int, steps: int) -> np.ndarray:
    """Estimates after each of the steps + 1 terms (array of length steps + 1)."""
    import scipy.sparse as sp

    w = np.ones(g.nnz) if g.w is None else g.w.astype(np.float64)
    A = sp.csr_matrix((w, g.col, g.row_ptr), shape=(g.n, g.n))
    d = np.asarray(A.sum(axis=1)).ravel()
    r = np.zeros(g.n)
    r[s] += 1.0
    r[t] -= 1.0
    rbar = 0.0
    out = np.empty(steps + 1)
    for i in range(steps + 1):
        rbar += r[s] / (2 * d[s]) - r[t] / (2 * d[t])
        out[i] = rbar
        r = 0.5 * r + 0.5 * (A @ (r / d))
    return out
