"""Seeded synthetic graph families and query-pair samplers.

Small closed-form families (complete, cycle, path, star, trees, the four-vertex
running example of Section 4.1) and the large stand-ins used for measurement:
a 2-D 4-neighbour grid (road-like, large condition number), a grid with random
edge deletions and uniform weights, Chung-Lu power-law graphs (social-like),
R-MAT, Erdos-Renyi and Barabasi-Albert. Every random choice comes from the
counter-based generator in ``graphgen.rng``; stream numbers are fixed per use
so a graph is a pure function of its parameters and seed.
"""
from __future__ import annotations

from typing import Optional

import numpy as np

from . import rng
from .graph import CSRGraph, largest_component, to_csr, unique_undirected  # noqa: F401

# Stream ids (arbitrary constants, one per independent use of randomness).
_S_CL_A, _S_CL_B = 11, 12
_S_DEL = 21
_S_W = 31
_S_PAIR_S, _S_PAIR_T = 41, 42
_S_RMAT = 51
_S_TREE = 61
_S_ER_U, _S_ER_V = 71, 72
_S_BA = 81
_S_GRIDPAIR = 91


def complete(n: int) -> CSRGraph:
    a, b = np.triu_indices(n, 1)
    return to_csr(n, a, b, name=f"K{n}")


def cycle(n: int) -> CSRGraph:
    a = np.arange(n)
    return to_csr(n, *unique_undirected(a, (a + 1) % n), name=f"C{n}")


def path(n: int) -> CSRGraph:
    a = np.arange(n - 1)
    return to_csr(n, a, a + 1, name=f"P{n}")


def star(n: int) -> CSRGraph:
    b = np.arange(1, n)
    return to_csr(n, np.zeros(n - 1, dtype=np.int64), b, name=f"S{n}")


def toy_graph() -> CSRGraph:
    """The four-vertex example of Section 4.1 with vertices 1..4 renumbered 0..3:
    edges (1,2), (1,3), (1,4), (2,3)."""
    a = np.array([0, 0, 0, 1])
    b = np.array([1, 2, 3, 2])
    return to_csr(4, a, b, name="toy4")


def random_tree(n: int, seed: int) -> CSRGraph:
    """Random recursive tree: vertex i > 0 attaches to a uniform earlier vertex."""
    parent = np.zeros(n, dtype=np.int64)
    if n > 1:
        u = rng.uniform(seed, _S_TREE, n - 1)
        parent[1:] = np.floor(u * np.arange(1, n)).astype(np.int64)
    child = np.arange(1, n)
    a, b = unique_undirected(parent[1:], child)
    g = to_csr(n, a, b, name=f"tree{n}")
    g.meta = {"parent": parent}
    return g


def grid(nx: int, ny: Optional[int] = None) -> CSRGraph:
    """nx-by-ny 4-neighbour grid; vertex (x, y) has id y*nx + x."""
    ny = nx if ny is None else ny
    ids = np.arange(nx * ny, dtype=np.int64).reshape(ny, nx)
    a = np.concatenate([ids[:, :-1].ravel(), ids[:-1, :].ravel()])
    b = np.concatenate([ids[:, 1:].ravel(), ids[1:, :].ravel()])
    g = to_csr(nx * ny, *_sorted_pairs(a, b), name=f"grid{nx}x{ny}")
    g.meta = {"nx": nx, "ny": ny}
    return g


def _sorted_pairs(a, b):
    order = np.lexsort((b, a))
    return a[order], b[order]


def uniform_edge_weights(m: int, lo: float, hi: float, seed: int) -> np.ndarray:
    return (lo + (hi - lo) * rng.uniform(seed, _S_W, m)).astype(np.float32)


def lognormal_edge_weights(m: int, mu: float, sigma: float, seed: int) -> np.ndarray:
    return np.exp(mu + sigma * rng.normal(seed, _S_W, m)).astype(np.float32)


def weighted(g: CSRGraph, w_und: np.ndarray) -> CSRGraph:
    """Attach one weight per undirected edge (in ``undirected_edges`` order)."""
    a, b, _ = g.undirected_edges()
    out = to_csr(g.n, a, b, w_und, g.name + "_w")
    out.meta = g.meta
    return out


def grid_deleted(nx: int, p_delete: float, seed: int, w_lo: float = 0.5, w_hi: float = 2.0) -> CSRGraph:
    """Road-like grid: each edge deleted with probability ``p_delete``, largest component kept
    (order-preserving relabel), weights uniform in [w_lo, w_hi] per undirected edge."""
    g = grid(nx)
    a, b, _ = g.undirected_edges()
    keep = rng.uniform(seed, _S_DEL, a.size) >= p_delete
    g2 = to_csr(g.n, a[keep], b[keep], name=f"grid{nx}del")
    g2.meta = {"nx": nx, "ny": nx}
    g3 = largest_component(g2)
    a3, b3, _ = g3.undirected_edges()
    w = uniform_edge_weights(a3.size, w_lo, w_hi, seed)
    out = to_csr(g3.n, a3, b3, w, g3.name)
    meta = dict(g3.meta or {})
    meta.update(nx=nx, ny=nx, p_delete=p_delete, seed=seed)
    if "lcc_old_id" not in meta:
        meta["lcc_old_id"] = np.arange(g.n, dtype=np.int64)
    out.meta = meta
    return out


def chung_lu_weights(n: int, gamma: float, mean_degree: float, iters: int = 50) -> np.ndarray:
    """Expected degrees w_i proportional to (i+1)^(-1/(gamma-1)), scaled to the mean degree and
    capped at sqrt(sum w) (cap and rescale repeated until stable)."""
    w = np.power(np.arange(1, n + 1, dtype=np.float64), -1.0 / (gamma - 1.0))
    w *= mean_degree * n / w.sum()
    for _ in range(iters):
        cap = np.sqrt(w.sum())
        w = np.minimum(w, cap)
        w *= mean_degree * n / w.sum()
    return w


def chung_lu(n: int, gamma: float, mean_degree: float, m0: int, seed: int) -> CSRGraph:
    """Chung-Lu graph: ``m0`` endpoint pairs drawn independently proportional to the expected
    degrees, then self-loops dropped, duplicates removed, largest component kept."""
    w = chung_lu_weights(n, gamma, mean_degree)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    chunk = 1 << 24
    aa, bb = [], []
    for off in range(0, m0, chunk):
        cnt = min(chunk, m0 - off)
        ua = rng.uniform(seed, _S_CL_A, cnt, off)
        ub = rng.uniform(seed, _S_CL_B, cnt, off)
        aa.append(np.minimum(np.searchsorted(cdf, ua, side="right"), n - 1))
        bb.append(np.minimum(np.searchsorted(cdf, ub, side="right"), n - 1))
    a, b = unique_undirected(np.concatenate(aa), np.concatenate(bb))
    g = to_csr(n, a, b, name=f"chunglu{n}_g{gamma}")
    g.meta = {"gamma": gamma, "mean_degree": mean_degree, "m0": m0, "seed": seed}
    out = largest_component(g)
    out.meta = dict(out.meta or {})
    out.meta.update(g.meta)
    return out


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int, fast: bool = True) -> CSRGraph:
    """R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004): each of edge_factor * 2^scale edges
    picks one of four quadrants per level with probabilities (a, b, c, 1-a-b-c). No noise and
    no vertex permutation; symmetrised, deduplicated, largest component kept. ``fast`` uses the
    C generator (same random streams, identical graph)."""
    n = 1 << scale
    if fast:
        from . import fast as FG

        u, v = FG.rmat_edges(scale, edge_factor * n, a, b, c, seed, _S_RMAT)
        row_ptr, col = FG.csr_from_edges(n, u, v)
        del u, v
        g = CSRGraph(n, row_ptr, col, None, f"rmat{scale}")
        g.meta = {"scale": scale, "edge_factor": edge_factor, "abc": (a, b, c), "seed": seed}
        out = largest_component(g)
        out.meta = dict(out.meta or {})
        out.meta.update(g.meta)
        return out
    m = edge_factor * n
    chunk = 1 << 22
    ab, abc = a + b, a + b + c
    us, vs = [], []
    for off in range(0, m, chunk):
        cnt = min(chunk, m - off)
        u = np.zeros(cnt, dtype=np.int64)
        v = np.zeros(cnt, dtype=np.int64)
        for lvl in range(scale):
            r = rng.uniform(seed, _S_RMAT + 1000 * lvl, cnt, off)
            row_bit = (r >= ab).astype(np.int64)
            col_bit = (((r >= a) & (r < ab)) | (r >= abc)).astype(np.int64)
            u = (u << 1) | row_bit
            v = (v << 1) | col_bit
        us.append(u)
        vs.append(v)
    a2, b2 = unique_undirected(np.concatenate(us), np.concatenate(vs))
    g = to_csr(n, a2, b2, name=f"rmat{scale}")
    g.meta = {"scale": scale, "edge_factor": edge_factor, "abc": (a, b, c), "seed": seed}
    out = largest_component(g)
    out.meta = dict(out.meta or {})
    out.meta.update(g.meta)
    return out


def erdos_renyi(n: int, m: int, seed: int) -> CSRGraph:
    """G(n, m)-style: m uniform endpoint pairs, deduplicated, largest component kept."""
    a = rng.integers(seed, _S_ER_U, m, n)
    b = rng.integers(seed, _S_ER_V, m, n)
    g = to_csr(n, *unique_undirected(a, b), name=f"er{n}")
    return largest_component(g)


def barabasi_albert(n: int, m_attach: int, seed: int, fast: bool = True) -> CSRGraph:
    """Preferential attachment: each new vertex links to ``m_attach`` endpoints drawn from the
    list of all earlier edge endpoints (plus a seed clique); duplicates dropped. ``fast`` uses
    the C generator (same draws, identical graph)."""
    m0 = m_attach + 1
    if fast:
        from . import fast as FG

        src, dst = FG.ba_edges(n, m_attach, seed, _S_BA)
        return to_csr(n, *unique_undirected(src, dst), name=f"ba{n}")
    a0, b0 = np.triu_indices(m0, 1)
    ends = list(np.concatenate([a0, b0]))
    src, dst = list(a0), list(b0)
    draws = rng.uniform(seed, _S_BA, (n - m0) * m_attach)
    k = 0
    for v in range(m0, n):
        L = len(ends)
        for _ in range(m_attach):
            t = ends[int(draws[k] * L)]
            k += 1
            src.append(v)
            dst.append(t)
        ends.extend(dst[-m_attach:])
        ends.extend([v] * m_attach)
    return to_csr(n, *unique_undirected(np.array(src), np.array(dst)), name=f"ba{n}")


def random_connected(n: int, extra_edges: int, seed: int, weights: Optional[str] = None) -> CSRGraph:
    """Random tree plus ``extra_edges`` uniform chords: small connected test graphs."""
    t = random_tree(n, seed)
    ta, tb, _ = t.undirected_edges()
    ea = rng.integers(seed, _S_ER_U, extra_edges, n)
    eb = rng.integers(seed, _S_ER_V, extra_edges, n)
    a, b = unique_undirected(np.concatenate([ta, ea]), np.concatenate([tb, eb]))
    w = None
    if weights == "uniform":
        w = uniform_edge_weights(a.size, 0.5, 2.0, seed)
    elif weights == "lognormal":
        w = lognormal_edge_weights(a.size, 0.0, 0.5, seed)
    return to_csr(n, a, b, w, name=f"rc{n}")


def random_pairs(n: int, count: int, seed: int):
    """``count`` (s, t) pairs, s and t uniform over [0, n) with s != t (requires n >= 2)."""
    s = rng.integers(seed, _S_PAIR_S, count, n)
    t = rng.integers(seed, _S_PAIR_T, count, n - 1)
    t = np.where(t >= s, t + 1, t)
    return s.astype(np.int32), t.astype(np.int32)


def grid_distance_pairs(g: CSRGraph, count: int, dist: int, seed: int):
    """Pairs on a (possibly thinned) grid at Manhattan distance ``dist``: s uniform over the kept
    vertices, t = s + (dx, dy) with |dx| + |dy| = dist (random split and signs), resampled
    until t lies inside the grid and in the kept component."""
    nx, ny = g.meta["nx"], g.meta["ny"]
    old = g.meta.get("lcc_old_id")
    if old is None:
        old = np.arange(g.n, dtype=np.int64)
    new_of_old = np.full(nx * ny, -1, dtype=np.int64)
    new_of_old[old] = np.arange(old.size)
    ss, tt = [], []
    ctr = 0
    while len(ss) < count:
        u = rng.uniform(seed, _S_GRIDPAIR, 4, ctr * 4)
        ctr += 1
        s_new = min(int(u[0] * g.n), g.n - 1)
        so = int(old[s_new])
        sx, sy = so % nx, so // nx
        dx = min(int(u[1] * (dist + 1)), dist)
        dy = dist - dx
        sgn = int(u[2] * 4)
        if sgn & 1:
            dx = -dx
        if sgn & 2:
            dy = -dy
        tx, ty = sx + dx, sy + dy
        if not (0 <= tx < nx and 0 <= ty < ny):
            continue
        t_new = int(new_of_old[ty * nx + tx])
        if t_new < 0:
            continue
        ss.append(s_new)
        tt.append(t_new)
    return np.array(ss, dtype=np.int32), np.array(tt, dtype=np.int32)
