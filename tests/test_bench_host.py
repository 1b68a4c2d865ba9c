"""Host-side helpers of bench.py (CPU only)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from graphgen import families as F  # noqa: E402


def test_condition_number_matches_a_dense_eigendecomposition():
    """kappa = 2/(1 - mu_2) from the deflated sparse eigensolver equals the one from all
    eigenvalues of the dense normalised adjacency, on a grid and a weighted random graph."""
    import bench

    for g in (F.grid(9, 7), F.random_connected(120, 300, 5, "lognormal")):
        mu2, kappa = bench.condition_number(g, tol=1e-12)
        A = np.zeros((g.n, g.n))
        w = np.ones(g.nnz) if g.w is None else g.w.astype(np.float64)
        A[g.rows(), g.col] = w
        isd = 1.0 / np.sqrt(A.sum(axis=1))
        lam = np.linalg.eigvalsh(isd[:, None] * A * isd[None, :])
        assert abs(lam[-1] - 1.0) < 1e-12
        assert abs(mu2 - lam[-2]) < 1e-9
        assert abs(kappa - 2.0 / (1.0 - lam[-2])) < 1e-6 * kappa


def test_host_info_names_the_machine():
    import bench

    h = bench.host_info()
    assert h["machine"] and h["nproc"] >= 1
