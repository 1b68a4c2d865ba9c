"""Pins for the oracle: closed forms, invariants, the paper's one exact printed value,
and planted mistakes that the pins must catch. CPU only.

Each pin is independent of the oracle's own arithmetic: circuit laws (series,
parallel, trees, Foster's theorem), exact spectra (complete graph, cycle, grid),
the structural identities of Proposition lanczos_guarantee and Lemma
lz_quadratic_err, and brute-force finite differences for the gradient.
"""
import os
import subprocess

import numpy as np
import pytest

from graphgen import families as F
from graphgen.graph import to_csr
from oracle import dense, lanczos, power
from tests import closed_forms as CF

HERE = os.path.dirname(os.path.abspath(__file__))


def load_toy_golden():
    edges, pairs = [], []
    with open(os.path.join(HERE, "golden", "toy_graph.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "edge":
                edges.append((int(tok[1]) - 1, int(tok[2]) - 1))
            elif tok[0] == "pair":
                pairs.append((int(tok[1]) - 1, int(tok[2]) - 1, float(tok[3])))
    a, b = zip(*edges)
    return to_csr(4, np.array(a), np.array(b)), pairs


# ---------------------------------------------------------------- dense part

@pytest.mark.parametrize("n", [3, 5, 8])
def test_dense_complete(n):
    D = dense.DenseRD.of(F.complete(n))
    s, t = np.triu_indices(n, 1)
    np.testing.assert_allclose(D.r(s, t), CF.complete_graph_r(n), rtol=1e-13)


@pytest.mark.parametrize("n", [5, 9, 12])
def test_dense_cycle(n):
    D = dense.DenseRD.of(F.cycle(n))
    for h in range(1, n):
        assert D.r(0, h)[0] == pytest.approx(CF.cycle_r(n, h), rel=1e-13)


def test_dense_path_and_toy_golden():
    D = dense.DenseRD.of(F.path(7))
    for i in range(7):
        for j in range(7):
            assert D.r(i, j)[0] == pytest.approx(abs(i - j), abs=1e-12)
    g, pairs = load_toy_golden()
    D = dense.DenseRD.of(g)
    for s, t, r in pairs:
        assert D.r(s, t)[0] == pytest.approx(r, rel=1e-13)
    # triangle 1-2-3 with pendant 4: r(1,2) = 1 || 2 = 2/3 and r(2,4) = 2/3 + 1
    assert D.r(0, 1)[0] == pytest.approx(CF.parallel(1.0, 2.0), rel=1e-13)
    assert D.r(1, 3)[0] == pytest.approx(CF.series(CF.parallel(1.0, 2.0), 1.0), rel=1e-13)


def test_dense_weighted_tree():
    n = 40
    t = F.random_tree(n, 5)
    parent = t.meta["parent"]
    w_child = F.uniform_edge_weights(n, 0.5, 2.0, 9)  # weight of edge (v, parent[v]) is w_child[v]
    a = np.minimum(parent[1:], np.arange(1, n))
    b = np.maximum(parent[1:], np.arange(1, n))
    g = to_csr(n, a, b, w_child[1:])
    D = dense.DenseRD.of(g)
    for s, tt in [(0, 39), (5, 17), (12, 3), (38, 39)]:
        assert D.r(s, tt)[0] == pytest.approx(CF.tree_r(parent, w_child, s, tt), rel=1e-12)


def test_dense_series_parallel_gadget():
    # s=0 and t=1 joined by path A (0-2-3-1, weights 2, 0.5, 4) and path B (0-4-1, weights 1, 3)
    a = np.array([0, 2, 1, 0, 1])
    b = np.array([2, 3, 3, 4, 4])
    w = np.array([2.0, 0.5, 4.0, 1.0, 3.0], dtype=np.float32)
    order = np.lexsort((b, a))
    g = to_csr(5, a[order], b[order], w[order])
    RA = CF.series(1 / 2.0, 1 / 0.5, 1 / 4.0)
    RB = CF.series(1 / 1.0, 1 / 3.0)
    assert dense.DenseRD.of(g).r(0, 1)[0] == pytest.approx(CF.parallel(RA, RB), rel=1e-12)


@pytest.mark.parametrize("weights", [None, "uniform", "lognormal"])
def test_dense_foster(weights):
    g = F.random_connected(60, 120, 3, weights)
    D = dense.DenseRD.of(g)
    a, b, w = g.undirected_edges()
    w = np.ones(a.size) if w is None else w.astype(np.float64)
    assert np.sum(w * D.r(a, b)) == pytest.approx(g.n - 1, rel=1e-11)


@pytest.mark.parametrize("nx,ny", [(8, 8), (5, 7)])
def test_dense_grid_spectral(nx, ny):
    g = F.grid(nx, ny)
    D = dense.DenseRD.of(g)
    for s, t in [(0, nx * ny - 1), (3, 17), (nx + 1, nx * ny - 2)]:
        assert D.r(s, t)[0] == pytest.approx(CF.grid_r(nx, ny, s, t), rel=1e-12)


def test_dense_gradient_fd_euler_rayleigh():
    g = F.random_connected(30, 40, 11, "lognormal")
    D = dense.DenseRD.of(g)
    s, t = np.array([0, 7, 3]), np.array([29, 21, 4])
    gbar = np.array([1.0, -0.5, 2.0])
    grad = D.edge_grad(s, t, gbar)
    rows = g.rows()
    # Euler: r is homogeneous of degree -1 in w, so sum_e w_e dr/dw_e = -r
    r = D.r(s, t)
    assert np.sum(g.w.astype(np.float64) * grad) == pytest.approx(-np.dot(gbar, r), rel=1e-10)
    # Rayleigh monotonicity (gbar > 0 only)
    assert np.all(D.edge_grad(s, t, np.abs(gbar)) <= 1e-15)
    # central finite differences on symmetric perturbations of both stored copies
    for e in [0, 5, 17, 40]:
        u, v = rows[e], g.col[e]
        e2 = np.nonzero((rows == v) & (g.col == u))[0][0]
        h = 1e-5 * float(g.w[e])
        def r_at(delta):
            ww = g.w.astype(np.float64).copy()
            ww[e] += delta
            ww[e2] += delta
            return np.dot(gbar, dense.DenseRD(g.n, g.row_ptr, g.col, ww).r(s, t))
        fd = (r_at(h) - r_at(-h)) / (2 * h)
        assert grad[e] + grad[e2] == pytest.approx(fd, rel=1e-6, abs=1e-12)
        assert grad[e] == pytest.approx(grad[e2], rel=1e-12)


# ------------------------------------------------------------- Lanczos part

def test_lanczos_complete_breaks_down_after_one_step():
    for n in [4, 6, 9]:
        out = lanczos.lanczos_pair(F.complete(n), 0, n - 1, k_max=10)
        assert out["k"] == 1
        assert out["alpha"][0] == pytest.approx(-1.0 / (n - 1), abs=1e-14)
        assert out["r"] == pytest.approx(CF.complete_graph_r(n), rel=1e-13)


@pytest.mark.parametrize("n,h", [(9, 3), (12, 6), (15, 1)])
def test_lanczos_cycle(n, h):
    out = lanczos.lanczos_pair(F.cycle(n), 0, h, k_max=n)
    assert out["r"] == pytest.approx(CF.cycle_r(n, h), rel=1e-12)


def test_lanczos_toy_golden_and_path():
    g, pairs = load_toy_golden()
    for s, t, r in pairs:
        assert lanczos.lanczos_pair(g, s, t, k_max=4)["r"] == pytest.approx(r, rel=1e-13)
    p = F.path(10)
    assert lanczos.lanczos_pair(p, 2, 9, k_max=10)["r"] == pytest.approx(7.0, rel=1e-12)


def test_lanczos_grid_spectral():
    g = F.grid(8)
    for s, t in [(0, 63), (9, 54), (1, 2)]:
        out = lanczos.lanczos_pair(g, s, t, k_max=200, stop_tol=1e-15)
        assert out["r"] == pytest.approx(CF.grid_r(8, 8, s, t), rel=1e-11)


def test_lanczos_grid64_corner_closed_form():
    """The 64x64 grid, corner to corner, FP64: the small measured workload."""
    g = F.grid(64)
    ref = CF.grid_r(64, 64, 0, 4095)
    out = lanczos.lanczos_pair(g, 0, 4095, k_max=500, stop_tol=1e-15)
    assert out["r"] == pytest.approx(ref, rel=1e-10)
    assert out["k"] < 500


@pytest.mark.parametrize("weights", [None, "uniform", "lognormal"])
def test_lanczos_vs_dense_random(weights):
    g = F.random_connected(80, 150, 21, weights)
    D = dense.DenseRD.of(g)
    s, t = F.random_pairs(g.n, 6, 4)
    r, k, _ = lanczos.lanczos_batch(g, s, t, k_max=200, stop_tol=1e-15, threads=2)
    np.testing.assert_allclose(r, D.r(s, t), rtol=1e-10)


def test_lanczos_relation_and_spectrum():
    """Proposition lanczos_guarantee: Ahat V_k = V_k T_k + beta_{k+1} v_{k+1} e_k^T,
    V_k orthonormal (small k), and Lemma lz_quadratic_err: eig(T_k) within
    [lambda_min(Ahat), lambda_2(Ahat)]; rhat_k = |b|^2 [(I - T_k)^{-1}]_{11}."""
    g = F.random_connected(50, 80, 8, "uniform")
    A = CF.normalized_adjacency(g.n, g.row_ptr, g.col, g.w)
    k = 8
    out = lanczos.lanczos_pair(g, 3, 41, k_max=k, want_basis=True)
    assert out["k"] == k
    V = out["V"]
    a, b = out["alpha"], out["beta"]
    T = np.diag(a) + np.diag(b[1:k], 1) + np.diag(b[1:k], -1)
    Vk = V[:, :k]
    resid = A @ Vk - Vk @ T
    resid[:, k - 1] -= b[k] * V[:, k]
    assert np.abs(resid).max() < 1e-13
    assert np.abs(Vk.T @ Vk - np.eye(k)).max() < 1e-12
    lam = np.linalg.eigvalsh(A)
    th = np.linalg.eigvalsh(T)
    assert th.min() >= lam[0] - 1e-12 and th.max() <= lam[-2] + 1e-12
    deg = np.zeros(g.n)
    np.add.at(deg, g.rows(), g.w.astype(np.float64))
    b2 = 1 / deg[3] + 1 / deg[41]
    e1 = np.zeros(k)
    e1[0] = 1.0
    assert out["r"] == pytest.approx(b2 * np.linalg.solve(np.eye(k) - T, e1)[0], rel=1e-13)


def test_lanczos_monotone_lower_bound_symmetry_scaling():
    g = F.grid_deleted(20, 0.05, 3)
    D = dense.DenseRD.of(g)
    s, t = 0, g.n - 1
    out = lanczos.lanczos_pair(g, s, t, k_max=60)
    h = out["r_hist"]
    assert np.all(np.diff(h) >= -1e-14 * h[-1])
    assert np.all(h <= D.r(s, t)[0] * (1 + 1e-13))
    r_ts = lanczos.lanczos_pair(g, t, s, k_max=60)["r"]
    assert r_ts == pytest.approx(out["r"], rel=1e-12)
    g2 = g.with_weights((2.0 * g.w).astype(np.float32))
    assert lanczos.lanczos_pair(g2, s, t, k_max=60)["r"] == pytest.approx(out["r"] / 2, rel=1e-13)
    assert lanczos.lanczos_pair(g, 5, 5, k_max=10)["r"] == 0.0


def test_lanczos_potential_matches_dense():
    g = F.random_connected(40, 70, 13, "lognormal")
    D = dense.DenseRD.of(g)
    out = lanczos.lanczos_pair(g, 2, 33, k_max=120, stop_tol=1e-15, want_potential=True)
    phi = out["phi"] - out["phi"].mean()
    ref = D.potential(2, 33)
    # r converges quadratically in the solve error, phi only linearly: looser bound here
    np.testing.assert_allclose(phi, ref - ref.mean(), atol=1e-8 * np.abs(ref).max())


def test_direct_potential_update_equals_algorithm5_potential():
    """The recurrence the CUDA path uses for the potential (built during the forward steps:
    with I - T_i = L D L^T, p_i = v_i + (beta_i/delta_{i-1}) p_{i-1} and
    x_i = x_{i-1} + ||b|| (g_i/delta_i) p_i) gives, at every k, Algorithm 5's
    ||b|| V_k (I - T_k)^{-1} e_1, and after D^{-1/2} the oracle's potential; checked here on
    the oracle's basis and coefficients, with the solve done afresh at each k."""
    g = F.random_connected(60, 120, 17, "lognormal")
    s, t, K = 4, 51, 25
    out = lanczos.lanczos_pair(g, s, t, k_max=K, want_basis=True)
    V, a, b = out["V"], out["alpha"], out["beta"]
    k = out["k"]
    assert k == K
    deg = np.zeros(g.n)
    np.add.at(deg, g.rows(), g.w.astype(np.float64))
    bn = np.sqrt(1 / deg[s] + 1 / deg[t])
    p = np.zeros(g.n)
    x = np.zeros(g.n)
    d_prev = g_prev = None
    for i in range(k):
        if i == 0:
            lam, d, gi = 0.0, 1.0 - a[0], 1.0
        else:
            lam = b[i] / d_prev
            d = (1.0 - a[i]) - b[i] ** 2 / d_prev
            gi = g_prev * b[i] / d_prev
        p = V[:, i] + lam * p
        x = x + bn * (gi / d) * p
        T = np.diag(a[:i + 1]) + np.diag(b[1:i + 1], 1) + np.diag(b[1:i + 1], -1)
        e1 = np.zeros(i + 1)
        e1[0] = 1.0
        ref = bn * V[:, :i + 1] @ np.linalg.solve(np.eye(i + 1) - T, e1)
        assert np.abs(x - ref).max() <= 1e-12 * np.abs(ref).max(), i
        d_prev, g_prev = d, gi
    phi = lanczos.lanczos_pair(g, s, t, k_max=K, want_potential=True)["phi"]
    assert np.abs(x / np.sqrt(deg) - phi).max() <= 1e-12 * np.abs(phi).max()


# ---------------------------------------------------- planted mistakes

MUTATIONS = {
    "v1_plus_sign": ("vcur[t] = -isd[t] / bnorm;", "vcur[t] = isd[t] / bnorm;"),
    "dropped_beta_term": ("u[x] = acc - b[i] * vprev[x];", "u[x] = acc;"),
    "norm_missing_dt": ("const double bnorm2 = 1.0 / deg[s] + 1.0 / deg[t];", "const double bnorm2 = 1.0 / deg[s];"),
    "wrong_scaling_index": ("acc += wv * isd[x] * isd[col[e]] * vcur[col[e]];", "acc += wv * isd[x] * isd[x] * vcur[col[e]];"),
    "alpha_not_subtracted": ("u[x] -= al * vcur[x];", "u[x] -= 0.0 * al * vcur[x];"),
    "thomas_sign": ("double lower = -b[j];", "double lower = b[j] * 0.5;"),
}


def _pins_pass(lib) -> bool:
    """A compact battery of the pins above, run against a given oracle build."""
    try:
        checks = []
        for n in [5, 8]:
            out = lanczos.lanczos_pair(F.complete(n), 0, n - 1, k_max=10, lib=lib)
            checks.append(abs(out["r"] - 2.0 / n) < 1e-10)
        out = lanczos.lanczos_pair(F.cycle(9), 0, 3, k_max=9, lib=lib)
        checks.append(abs(out["r"] - 2.0) < 1e-10)
        out = lanczos.lanczos_pair(F.grid(8), 0, 63, k_max=200, stop_tol=1e-15, lib=lib)
        checks.append(abs(out["r"] / CF.grid_r(8, 8, 0, 63) - 1) < 1e-9)
        g = F.star(6)
        out = lanczos.lanczos_pair(g, 1, 2, k_max=6, lib=lib)
        checks.append(abs(out["r"] - 2.0) < 1e-10)
        return all(checks)
    except Exception:
        return False


def test_pins_pass_unmutated():
    assert _pins_pass(lanczos.load())


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(os.path.join(os.path.dirname(lanczos.__file__), "lanczos_ref.c")).read()
    assert src.count(old) == 1, f"mutation anchor not found: {old}"
    mut = tmp_path / f"{name}.c"
    mut.write_text(src.replace(old, new))
    so = str(tmp_path / f"lib{name}.so")
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", so, str(mut), "-lm"])
    assert not _pins_pass(lanczos.load(so)), f"planted mistake {name} passed every pin"


# ------------------------------------------------------- Power Method part

@pytest.mark.parametrize("make,s,t,ref", [
    (lambda: F.complete(6), 0, 5, 2.0 / 6),
    (lambda: F.cycle(10), 0, 4, CF.cycle_r(10, 4)),
    (lambda: F.grid(6), 0, 35, CF.grid_r(6, 6, 0, 35)),
])
def test_power_method_converges_to_closed_forms(make, s, t, ref):
    """Algorithm 1 is the series of Eq. (er_laylor_expansion): increasing partial sums
    (each term is nonnegative) that converge to r."""
    h = power.power_method(make(), s, t, 4000)
    assert h[-1] == pytest.approx(ref, rel=1e-10)
    assert np.all(np.diff(h) >= -1e-15)


def test_power_method_first_terms_by_hand():
    """Path 0-1-2 (degrees 1, 2, 1), s=0, t=2: r_0 = e_0 - e_2 gives term 1/2 + 1/2 = 1; then
    r_1 = (I/2 + P/2) r_0 = [1/2, 0, -1/2] gives 1/4 + 1/4 = 1/2."""
    h = power.power_method(F.path(3), 0, 2, 2)
    assert h[0] == pytest.approx(1.0, abs=1e-15)
    assert h[1] == pytest.approx(1.5, abs=1e-15)


def _laplacian_cg_r(g, s, t):
    """r(s,t) from an independent solver: Jacobi-preconditioned conjugate gradients (scipy)
    on L phi = e_s - e_t (consistent: the right-hand side sums to zero), r = phi_s - phi_t."""
    import scipy.sparse as sp
    from scipy.sparse.linalg import LinearOperator, cg

    w = np.ones(g.nnz) if g.w is None else g.w.astype(np.float64)
    A = sp.csr_matrix((w, g.col, g.row_ptr), shape=(g.n, g.n))
    d = np.asarray(A.sum(axis=1)).ravel()
    L = sp.diags(d) - A
    b = np.zeros(g.n)
    b[s] += 1.0
    b[t] -= 1.0
    M = LinearOperator((g.n, g.n), matvec=lambda x: x / d)
    try:
        phi, info = cg(L, b, rtol=1e-14, atol=0.0, maxiter=200000, M=M)
    except TypeError:  # older scipy spells the tolerance `tol`
        phi, info = cg(L, b, tol=1e-14, atol=0.0, maxiter=200000, M=M)
    assert info == 0
    return phi[s] - phi[t]


@pytest.mark.parametrize("family", ["chunglu", "grid_weighted", "ba"])
def test_lanczos_vs_independent_cg_at_scale(family):
    """Sizes where the dense pseudo-inverse is out of reach: the FP64 Lanczos oracle, run to a
    1e-15 relative increment, agrees with Jacobi-CG on the Laplacian to 1e-9 relative."""
    from graphgen import workloads as W

    if family == "chunglu":
        g, s, t = W.chunglu(20000, 2.1, 20.0, 200000, 4, 19)
    elif family == "grid_weighted":
        g = F.grid_deleted(90, 0.05, 4)
        s, t = F.random_pairs(g.n, 4, 6)
    else:
        g = F.barabasi_albert(15000, 3, 8)
        s, t = F.random_pairs(g.n, 4, 7)
    for a, b in zip(s, t):
        r_lz = lanczos.lanczos_pair(g, int(a), int(b), k_max=20000, stop_tol=1e-15)["r"]
        r_cg = _laplacian_cg_r(g, int(a), int(b))
        assert abs(r_lz - r_cg) / r_cg < 1e-9, (family, a, b, r_lz, r_cg)
