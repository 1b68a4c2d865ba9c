#!/usr/bin/env python3
"""Write tests/golden/roadgrid1024_ref.json: converged reference values of r(s,t) on a
road-like grid small enough for the CPU oracle.

Graph: 1024 x 1024 4-neighbour grid, each edge deleted with probability 0.05 (seed 11),
largest component, weights uniform in [0.5, 2.0] (graphgen.families.grid_deleted);
8 pairs at Manhattan distance 256 (graphgen.families.grid_distance_pairs, seed 5).

Values: the FP64 oracle (Algorithm 3 verbatim, oracle/lanczos_ref.c) run to a relative
increment of 1e-13, on every pair; cross-checked on two pairs by an independent solver,
Jacobi-preconditioned conjugate gradients on L phi = e_s - e_t (scipy), which must agree to
1e-9 relative before anything is written. Nothing here touches the CUDA library.

Run from the repository root: python tests/golden/make_roadgrid1024_ref.py
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from graphgen import families as F  # noqa: E402
from oracle import lanczos  # noqa: E402

NX, P_DELETE, SEED, PAIRS, DIST, PAIR_SEED = 1024, 0.05, 11, 8, 256, 5
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "roadgrid1024_ref.json")


def graph_and_pairs():
    g = F.grid_deleted(NX, P_DELETE, SEED)
    s, t = F.grid_distance_pairs(g, PAIRS, DIST, PAIR_SEED)
    return g, s, t


def checksum(g) -> str:
    h = hashlib.sha1()
    for a in (g.row_ptr, g.col, g.w):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def cg_r(g, s, t):
    import scipy.sparse as sp
    from scipy.sparse.linalg import LinearOperator, cg

    A = sp.csr_matrix((g.w.astype(np.float64), g.col, g.row_ptr), shape=(g.n, g.n))
    d = np.asarray(A.sum(axis=1)).ravel()
    L = sp.diags(d) - A
    b = np.zeros(g.n)
    b[s] += 1.0
    b[t] -= 1.0
    M = LinearOperator((g.n, g.n), matvec=lambda x: x / d)
    try:
        phi, info = cg(L, b, rtol=1e-14, atol=0.0, maxiter=400000, M=M)
    except TypeError:  # older scipy spells the tolerance `tol`
        phi, info = cg(L, b, tol=1e-14, atol=0.0, maxiter=400000, M=M)
    assert info == 0, info
    return float(phi[s] - phi[t])


def main():
    g, s, t = graph_and_pairs()
    t0 = time.time()
    r, k, threads = lanczos.lanczos_batch(g, s, t, k_max=100000, stop_tol=1e-13, threads=0)
    t1 = time.time()
    checks = []
    for i in (0, PAIRS - 1):
        rc = cg_r(g, int(s[i]), int(t[i]))
        rel = abs(r[i] - rc) / rc
        assert rel < 1e-9, (i, r[i], rc, rel)
        checks.append({"pair": i, "r_cg": rc, "rel_diff": rel})
    out = {
        "graph": {"nx": NX, "p_delete": P_DELETE, "seed": SEED, "n": g.n, "nnz": g.nnz, "sha1": checksum(g)},
        "pairs": {"count": PAIRS, "dist": DIST, "seed": PAIR_SEED, "s": s.tolist(), "t": t.tolist()},
        "oracle": {"stop": "relative increment 1e-13", "r": [float(x) for x in r], "k": [int(x) for x in k]},
        "cg_check": checks,
        "seconds": {"oracle": round(t1 - t0, 1), "threads": int(threads)},
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out["oracle"]), checks)


if __name__ == "__main__":
    main()
