"""Input generators: determinism and agreement of the C and numpy paths (CPU)."""
import numpy as np

from graphgen import families as F
from graphgen import rng


def test_rng_is_counter_based_and_sliceable():
    a = rng.uniform(7, 3, 100)
    b = rng.uniform(7, 3, 40, offset=60)
    assert np.array_equal(a[60:], b)
    assert a.min() >= 0.0 and a.max() < 1.0
    assert not np.array_equal(a, rng.uniform(7, 4, 100))


def test_rmat_c_generator_matches_numpy():
    g1 = F.rmat(10, 8, 0.57, 0.19, 0.19, 5, fast=True)
    g2 = F.rmat(10, 8, 0.57, 0.19, 0.19, 5, fast=False)
    assert g1.n == g2.n
    assert np.array_equal(g1.row_ptr, g2.row_ptr)
    assert np.array_equal(g1.col, g2.col)


def test_csr_is_symmetric_simple_connected():
    g = F.chung_lu(3000, 2.1, 10.0, 15000, 3)
    rows = g.rows()
    assert np.all(rows != g.col)
    key = rows * g.n + g.col
    assert np.unique(key).size == key.size
    back = np.sort(g.col.astype(np.int64) * g.n + rows)
    assert np.array_equal(np.sort(key), back)
    from graphgen.graph import component_labels

    assert np.unique(component_labels(g)).size == 1


def test_ba_c_generator_matches_python():
    a = F.barabasi_albert(3000, 5, 9, fast=True)
    b = F.barabasi_albert(3000, 5, 9, fast=False)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col)
