"""Plain CSR container and edge-list -> symmetric CSR assembly.

Input preparation only: dropping self-loops, removing duplicate undirected
edges, keeping the largest connected component with an order-preserving
relabel, and writing both stored copies (u, v) and (v, u) of every edge with
the same weight. Degrees and every other quantity of the method are left to
the code under test and to the oracle, each of which computes them itself.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np


@dataclass
class CSRGraph:
    """Symmetric CSR: ``row_ptr`` int64[n+1], ``col`` int32[nnz], ``w`` float32[nnz] or None."""

    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    w: Optional[np.ndarray] = None
    name: str = ""
    meta: Optional[dict] = None

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def m(self) -> int:
        return self.nnz // 2

    def rows(self) -> np.ndarray:
        """Row index of every stored entry (int64[nnz])."""
        return np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.row_ptr))

    def undirected_edges(self):
        """(u, v, w) with u < v, one entry per undirected edge, in CSR order."""
        r = self.rows()
        keep = r < self.col
        w = None if self.w is None else self.w[keep]
        return r[keep], self.col[keep].astype(np.int64), w

    def with_weights(self, w: Optional[np.ndarray]) -> "CSRGraph":
        return CSRGraph(self.n, self.row_ptr, self.col, w, self.name, self.meta)


def unique_undirected(u: np.ndarray, v: np.ndarray):
    """Drop self-loops and duplicates; return (a, b) with a < b, sorted by (a, b)."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    keep = u != v
    a = np.minimum(u[keep], v[keep])
    b = np.maximum(u[keep], v[keep])
    if a.size == 0:
        return a, b
    hi = int(b.max()) + 1
    key = np.unique(a * hi + b)
    return key // hi, key % hi


def to_csr(n: int, a: np.ndarray, b: np.ndarray, w: Optional[np.ndarray] = None, name: str = "") -> CSRGraph:
    """Symmetric CSR from unique undirected edges (a, b), columns sorted within rows."""
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    rows = np.concatenate([a, b])
    cols = np.concatenate([b, a])
    order = np.lexsort((cols, rows))
    rows = rows[order]
    cols = cols[order]
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    ww = None
    if w is not None:
        w = np.asarray(w, dtype=np.float32)
        ww = np.concatenate([w, w])[order]
    return CSRGraph(n, row_ptr, cols.astype(np.int32), ww, name)


def component_labels(g: CSRGraph) -> np.ndarray:
    """Connected-component label per vertex (scipy's BFS labelling)."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components

    mat = sp.csr_matrix((np.ones(g.nnz, dtype=np.int8), g.col, g.row_ptr), shape=(g.n, g.n))
    _, labels = connected_components(mat, directed=False)
    return labels


def largest_component(g: CSRGraph) -> CSRGraph:
    """Induced subgraph on the largest connected component, vertex order preserved.

    A component is closed under adjacency, so the kept rows keep all their entries; the
    relabelling is monotone, so rows and columns stay sorted without re-sorting."""
    labels = component_labels(g)
    counts = np.bincount(labels)
    big = int(np.argmax(counts))
    keep = labels == big
    if keep.all():
        return g
    new_id = np.cumsum(keep, dtype=np.int64) - 1
    deg = np.diff(g.row_ptr)
    entry_keep = np.repeat(keep, deg)
    n2 = int(keep.sum())
    row_ptr = np.zeros(n2 + 1, dtype=np.int64)
    np.cumsum(deg[keep], out=row_ptr[1:])
    col = new_id[g.col[entry_keep]].astype(np.int32)
    w = None if g.w is None else g.w[entry_keep]
    out = CSRGraph(n2, row_ptr, col, w, g.name)
    out.meta = dict(g.meta or {})
    out.meta["lcc_dropped_vertices"] = int(g.n - out.n)
    out.meta["lcc_old_id"] = np.nonzero(keep)[0]
    return out
