"""The named synthetic workloads (graph + query pairs), with on-disk caching.

Each workload fixes the graph family, its size, its seed and the query pairs:

* ``grid64``     -- 64x64 4-neighbour grid, unweighted, one pair: corner 0 to corner 4095.
* ``chunglu1m``  -- Chung-Lu, n = 1,000,000, exponent 2.1, mean degree 20, 1e7 endpoint draws,
                    largest component, unweighted; 256 uniform pairs.
* ``roadgrid4096`` -- 4096x4096 grid, 5% of edges deleted, largest component, weights
                    U[0.5, 2.0]; 64 pairs at Manhattan distance 1000.
* ``chunglu4m_w`` -- Chung-Lu, n = 4,000,000, exponent 2.3, mean degree 20, 4e7 draws,
                    lognormal(0, 0.5) weights; 32 pairs.
* ``rmat24``     -- R-MAT scale 24, edge factor 16, (a, b, c) = (0.57, 0.19, 0.19), largest
                    component, unweighted; 128 pairs.

A scaled-down variant of each family (``scale`` argument) serves the tests.
"""
from __future__ import annotations

import hashlib
import os
from typing import Optional, Tuple

import numpy as np

from . import families as F
from .graph import CSRGraph

BASE_SEED = 20260101


def cache_dir() -> str:
    """Where generated workload graphs are kept between runs: $RD_GRAPH_CACHE, else the
    repository's own .graph_cache/ (not versioned)."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    d = os.environ.get("RD_GRAPH_CACHE", os.path.join(root, ".graph_cache"))
    os.makedirs(d, exist_ok=True)
    return d


def _cached(key: str, build):
    path = os.path.join(cache_dir(), hashlib.sha1(key.encode()).hexdigest()[:16] + ".npz")
    if os.path.exists(path):
        z = np.load(path, allow_pickle=False)
        w = z["w"] if z["has_w"] else None
        meta = {k[5:]: (z[k] if z[k].ndim else z[k].item()) for k in z.files if k.startswith("meta_")}
        return CSRGraph(int(z["n"]), z["row_ptr"], z["col"], w, str(z["name"]), meta)
    g = build()
    meta = {}
    for k, v in (g.meta or {}).items():
        if isinstance(v, (int, float, np.ndarray, np.integer, np.floating)):
            meta["meta_" + k] = np.asarray(v)
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, n=g.n, row_ptr=g.row_ptr, col=g.col, w=g.w if g.w is not None else np.zeros(0, np.float32),
             has_w=g.w is not None, name=g.name, **meta)
    os.replace(tmp, path)
    return g


def grid64() -> Tuple[CSRGraph, np.ndarray, np.ndarray]:
    g = F.grid(64)
    return g, np.array([0], dtype=np.int32), np.array([64 * 64 - 1], dtype=np.int32)


def chunglu(n: int = 1_000_000, gamma: float = 2.1, mean_degree: float = 20.0, m0: Optional[int] = None,
            pairs: int = 256, seed: int = BASE_SEED + 2, weights: Optional[str] = None):
    m0 = int(n * mean_degree / 2) if m0 is None else m0
    key = f"chunglu:{n}:{gamma}:{mean_degree}:{m0}:{seed}:{weights}"

    def build():
        g = F.chung_lu(n, gamma, mean_degree, m0, seed)
        if weights == "lognormal":
            a, _, _ = g.undirected_edges()
            g = F.weighted(g, F.lognormal_edge_weights(a.size, 0.0, 0.5, seed))
        return g

    g = _cached(key, build)
    s, t = F.random_pairs(g.n, pairs, seed)
    return g, s, t


def chunglu1m(pairs: int = 256):
    return chunglu(1_000_000, 2.1, 20.0, 10_000_000, pairs, BASE_SEED + 2)


def chunglu4m_w(pairs: int = 32):
    return chunglu(4_000_000, 2.3, 20.0, 40_000_000, pairs, BASE_SEED + 4, weights="lognormal")


def roadgrid(nx: int = 4096, pairs: int = 64, dist: int = 1000, seed: int = BASE_SEED + 3):
    key = f"roadgrid:{nx}:0.05:{seed}"
    g = _cached(key, lambda: F.grid_deleted(nx, 0.05, seed))
    g.meta = dict(g.meta or {})
    g.meta.setdefault("nx", nx)
    g.meta.setdefault("ny", nx)
    s, t = F.grid_distance_pairs(g, pairs, dist, seed)
    return g, s, t


def roadgrid4096(pairs: int = 64):
    return roadgrid(4096, pairs, 1000, BASE_SEED + 3)


def rmat(scale: int = 24, pairs: int = 128, seed: int = BASE_SEED + 5):
    key = f"rmat:{scale}:16:0.57:0.19:0.19:{seed}"
    g = _cached(key, lambda: F.rmat(scale, 16, 0.57, 0.19, 0.19, seed))
    s, t = F.random_pairs(g.n, pairs, seed)
    return g, s, t


def rmat24(pairs: int = 128):
    return rmat(24, pairs)
