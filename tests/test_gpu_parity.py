"""GPU parity: the CUDA path (called through the C ABI via the thin binding) against
the CPU oracle on the same seeded inputs.

Tolerances: FP64 mode within 1e-9 relative of the oracle, FP32-vector mode within
1e-5 relative (the bars fixed for this method's two precision modes).
"""
import numpy as np
import pytest

from graphgen import families as F
from graphgen import workloads as W
from graphgen.graph import to_csr
from oracle import dense, lanczos, power
from tests import closed_forms as CF

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def rd():
    import torch

    assert torch.cuda.is_available()
    import paper_2601_11159_gb300 as rd

    rd.lib()  # fails loudly if the library is not built
    return rd


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / np.abs(b)


SMALL = [
    ("K7", lambda: F.complete(7)),
    ("C11", lambda: F.cycle(11)),
    ("P9", lambda: F.path(9)),
    ("toy", lambda: F.toy_graph()),
    ("grid8", lambda: F.grid(8)),
    ("grid5x7", lambda: F.grid(5, 7)),
    ("rc60u", lambda: F.random_connected(60, 100, 3, None)),
    ("rc70w", lambda: F.random_connected(70, 140, 5, "uniform")),
    ("rc80ln", lambda: F.random_connected(80, 200, 7, "lognormal")),
]


@pytest.mark.parametrize("name,make", SMALL)
@pytest.mark.parametrize("mode", ["fp64", "fp32"])
@pytest.mark.parametrize("kernel", ["group", "group_sorted", "stream", "async", "onchip"])
def test_small_graphs_vs_dense(rd, name, make, mode, kernel):
    g = make()
    s, t = F.random_pairs(g.n, 9, 17)
    ref = dense.DenseRD.of(g).r(s, t)
    G = rd.Graph.from_csr(g)
    tol = FP64_TOL if mode == "fp64" else FP32_TOL
    kw = dict(onchip=True) if kernel == "onchip" else dict(kernel=kernel, onchip=False)
    res = G.query(s, t, mode=mode, k_max=400, rel_tol=0.0, resid_tol=1e-12 if mode == "fp64" else 1e-6, **kw)
    assert np.all(res.status >= 0), res.status
    assert rel(res.r, ref).max() < tol, (name, mode, rel(res.r, ref).max())


@pytest.mark.parametrize("mode,tol", [("fp64", 1e-11), ("fp32", 2e-5)])
def test_fixed_k_matches_oracle_history(rd, mode, tol):
    """Same k, same recurrence: the GPU estimate after k steps equals the oracle's rhat_k."""
    g = F.grid_deleted(24, 0.05, 9)
    s, t = F.random_pairs(g.n, 5, 2)
    G = rd.Graph.from_csr(g)
    for k in [1, 2, 5, 12, 30]:
        ref = np.array([lanczos.lanczos_pair(g, int(a), int(b), k_max=k)["r"] for a, b in zip(s, t)])
        for onchip in (False, True):
            res = G.query(s, t, mode=mode, k_max=k, fixed_k=True, onchip=onchip)
            assert np.all(res.iters == k)
            assert rel(res.r, ref).max() < tol, (k, onchip, rel(res.r, ref).max())


def test_grid64_corner_fp64_closed_form(rd):
    """64x64 grid, s = 0, t = 4095, FP64, k <= 500 or relative residual 1e-10."""
    g, s, t = W.grid64()
    ref = CF.grid_r(64, 64, 0, 4095)
    G = rd.Graph.from_csr(g)
    res = G.query(s, t, mode="fp64", k_max=500, rel_tol=0.0, resid_tol=1e-10)
    assert res.status[0] == 0 and res.iters[0] < 500
    assert rel(res.r, [ref]).max() < FP64_TOL
    # the same with the single-vector SpMV paths (row-group and row-stream kernels)
    for kernel in ["group", "group_sorted", "stream"]:
        res1 = G.query(s, t, mode="fp64", k_max=500, rel_tol=0.0, resid_tol=1e-10, plain=True, kernel=kernel)
        assert rel(res1.r, [ref]).max() < FP64_TOL


def test_ragged_batch_edge_cases(rd):
    g = F.random_connected(300, 500, 4, "uniform")
    n = g.n
    s, t = F.random_pairs(n, 37, 8)          # 37 pairs: not a multiple of any tile
    s[3] = t[3]                              # s == t
    s[10], t[10] = 0, n - 1                  # extreme ids
    ref = dense.DenseRD.of(g).r(s, t)
    G = rd.Graph.from_csr(g)
    for mode, tol in [("fp64", FP64_TOL), ("fp32", FP32_TOL)]:
        for onchip in (False, True):
            res = G.query(s, t, mode=mode, rel_tol=0.0, resid_tol=1e-12 if mode == "fp64" else 1e-6, onchip=onchip)
            assert res.r[3] == 0.0 and res.iters[3] == 0 and res.status[3] == 0
            m = np.arange(37) != 3
            assert rel(res.r[m], ref[m]).max() < tol
    empty = G.query(np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert empty.r.size == 0


def test_disconnected_and_invalid(rd):
    a = F.cycle(6)
    b = F.path(5)
    ea, eb, _ = a.undirected_edges()
    fa, fb, _ = b.undirected_edges()
    g = to_csr(11, np.concatenate([ea, fa + 6]), np.concatenate([eb, fb + 6]))
    G = rd.Graph.from_csr(g)
    assert G.ncomponents == 2
    res = G.query(np.array([0, 6, 1], np.int32), np.array([3, 10, 8], np.int32), mode="fp64", rel_tol=1e-12)
    assert res.r[0] == pytest.approx(CF.cycle_r(6, 3), rel=1e-9)
    assert res.r[1] == pytest.approx(4.0, rel=1e-9)
    assert np.isinf(res.r[2]) and res.status[2] == rd.RD_ERR_DISCONNECTED
    with pytest.raises(rd.RDError):
        G.query(np.array([0], np.int32), np.array([11], np.int32))
    with pytest.raises(rd.RDError):
        G.query(np.array([-1], np.int32), np.array([2], np.int32))


def test_bad_graphs_rejected(rd):
    g = F.path(4)
    with pytest.raises(rd.RDError):
        rd.Graph(g.row_ptr, np.array([1, 0, 2, 1, 3, 9], np.int32))           # column out of range
    with pytest.raises(rd.RDError):
        rd.Graph(g.row_ptr, g.col, np.array([1, 1, -1, 1, 1, 1], np.float32))  # negative weight
    with pytest.raises(rd.RDError):
        rd.Graph(np.array([0, 1, 2, 2], np.int64), np.array([1, 0], np.int32))  # isolated vertex 2
    asym = to_csr(3, np.array([0, 1]), np.array([1, 2]), np.array([1.0, 2.0], np.float32))
    w = asym.w.copy()
    w[0] = 5.0
    with pytest.raises(rd.RDError):
        rd.Graph(asym.row_ptr, asym.col, w, check_symmetry=True)


def test_self_loops_dropped(rd):
    g = F.random_connected(40, 60, 2, "uniform")
    rows = g.rows()
    # insert a self-loop at every vertex
    ra = np.concatenate([rows, np.arange(g.n)])
    ca = np.concatenate([g.col.astype(np.int64), np.arange(g.n)])
    wa = np.concatenate([g.w, np.full(g.n, 3.0, np.float32)])
    order = np.lexsort((ca, ra))
    rp = np.zeros(g.n + 1, np.int64)
    np.cumsum(np.bincount(ra, minlength=g.n), out=rp[1:])
    G = rd.Graph(rp, ca[order].astype(np.int32), wa[order])
    assert G.nnz == g.nnz
    s, t = F.random_pairs(g.n, 5, 1)
    res = G.query(s, t, mode="fp64", rel_tol=0.0, resid_tol=1e-12)
    assert rel(res.r, dense.DenseRD.of(g).r(s, t)).max() < FP64_TOL


@pytest.mark.parametrize("mode,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
@pytest.mark.parametrize("kernel", ["group", "group_sorted", "stream"])
def test_batched_vs_plain_and_order(rd, mode, tol, kernel):
    g, s, t = W.chunglu(20000, 2.1, 20.0, 200000, 40, 77)
    G = rd.Graph.from_csr(g)
    kw = dict(mode=mode, k_max=60, fixed_k=True, kernel=kernel)
    b = G.query(s, t, **kw)
    p = G.query(s, t, plain=True, **kw)
    assert rel(b.r, p.r).max() < tol
    for tile in [16, 32, 64, 128, 256]:
        if mode == "fp64" and tile == 256:
            continue
        bt = G.query(s, t, rhs_tile=tile, **kw)
        assert rel(bt.r, p.r).max() < tol, tile
    perm = np.random.default_rng(0).permutation(len(s))
    bp = G.query(s[perm], t[perm], **kw)
    assert np.array_equal(bp.r, b.r[perm])      # same batch size: bitwise equal per pair
    again = G.query(s, t, **kw)
    assert np.array_equal(again.r, b.r)          # deterministic


@pytest.mark.parametrize("weighted", [False, True])
def test_async_kernel_vs_oracle_and_row_stream(rd, weighted):
    """The row-stream SpMM with asynchronous gathers into a shared-memory ring (FP32 vectors):
    on a power-law graph with heavy rows (split into chunks by the pre-pass) and a ragged pair
    count, every column slab width agrees with the oracle at convergence, with the row-stream
    kernel at fixed k, and with itself bitwise on a repeat and under a permutation; new
    weights are followed."""
    kernel = "async"
    g, s, t = W.chunglu(20000, 2.1, 20.0, 200000, 37, 77, weights="lognormal" if weighted else None)
    assert np.diff(g.row_ptr).max() > 256  # heavy rows present
    G = rd.Graph.from_csr(g)
    ref, _, _ = lanczos.lanczos_batch(g, s, t, k_max=300, stop_tol=1e-14, threads=0)
    code = 5
    for tile in [16, 32, 64, 128]:
        kw = dict(mode="fp32", kernel=kernel, rhs_tile=tile, compact=False)
        res = G.query(s, t, k_max=300, rel_tol=0.0, resid_tol=1e-7, **kw)
        st = G.last_stats()
        assert st["kernel"] == code and st["rhs_tile"] == tile
        assert np.all(res.status >= 0)
        assert rel(res.r, ref).max() < FP32_TOL, (tile, rel(res.r, ref).max())
        fa = G.query(s, t, k_max=25, fixed_k=True, **kw)
        fs = G.query(s, t, mode="fp32", kernel="stream", rhs_tile=tile, compact=False, k_max=25, fixed_k=True)
        assert rel(fa.r, fs.r).max() < 2e-6, (tile, rel(fa.r, fs.r).max())
        assert np.array_equal(G.query(s, t, k_max=25, fixed_k=True, **kw).r, fa.r)
        perm = np.random.default_rng(1).permutation(len(s))
        fp = G.query(s[perm], t[perm], k_max=25, fixed_k=True, **kw)
        assert np.array_equal(fp.r, fa.r[perm])
    # graph replay and the compacting default path with this kernel
    kw = dict(mode="fp32", kernel=kernel, rhs_tile=32, k_max=300, rel_tol=1e-7)
    a = G.query(s, t, **kw)
    b = G.query(s, t, graph=False, **kw)
    assert np.array_equal(a.r, b.r)
    assert rel(a.r, ref).max() < FP32_TOL
    # new weights: the next query follows them
    w2 = F.lognormal_edge_weights(g.m, 0.0, 0.7, 91)
    g2 = F.weighted(g, w2)
    G.set_weights(g2.w)
    ref2, _, _ = lanczos.lanczos_batch(g2, s, t, k_max=300, stop_tol=1e-14, threads=0)
    r2 = G.query(s, t, mode="fp32", kernel=kernel, rhs_tile=64, compact=False, k_max=300, rel_tol=0.0,
                 resid_tol=1e-7).r
    assert rel(r2, ref2).max() < FP32_TOL


def _weakly_coupled(kind: str, eps: float):
    """Cliques joined through one edge of weight eps: the Krylov space of a pair across the
    weak edge is nearly invariant at some step, where beta_{i+1} / (|alpha_i| + beta_i)
    falls to 1e-5 .. 1e-8 before the recurrence goes on."""
    parts = [F.complete(40), F.path(10), F.complete(40)] if kind == "K40-P10-K40" else [F.complete(50), F.path(8)]
    links = [(0, 0, 1, 0, eps), (1, 9, 2, 0, 1.0)] if kind == "K40-P10-K40" else [(0, 0, 1, 0, eps)]
    off, A, B, Wt, offs = 0, [], [], [], []
    for g in parts:
        a, b, _ = g.undirected_edges()
        A.append(a + off)
        B.append(b + off)
        Wt.append(np.ones(a.size))
        offs.append(off)
        off += g.n
    for i, u, j, v, w in links:
        A.append(np.array([offs[i] + u]))
        B.append(np.array([offs[j] + v]))
        Wt.append(np.array([w]))
    g = to_csr(off, np.concatenate(A), np.concatenate(B), np.concatenate(Wt).astype(np.float32))
    pairs = [(1, 55), (3, 45)] if kind == "K40-P10-K40" else [(1, 57), (4, 52)]
    return g, np.array([p[0] for p in pairs], np.int32), np.array([p[1] for p in pairs], np.int32)


@pytest.mark.parametrize("kind,eps", [("K40-P10-K40", 1e-2), ("K40-P10-K40", 1e-3), ("K50+P8", 1e-2),
                                      ("K50+P8", 1e-3)])
def test_near_invariant_krylov_steps(rd, kind, eps):
    """Steps where beta_{i+1} is tiny against alpha_i (the cancellation regime of
    beta_{i+1}^2 = ||w||^2 - alpha_i^2 - gamma^2): the FP64 and double-float paths follow the
    oracle's r_k history at fixed k and converge to the dense pseudo-inverse value. The
    tolerance is 1e-8, above the FP64 oracle's own error on these graphs (up to 2.5e-9 against
    the dense reference: the weak edge makes them ill-conditioned)."""
    g, s, t = _weakly_coupled(kind, eps)
    ref = dense.DenseRD.of(g).r(s, t)
    # the regime is reached: beta_{i+1} / (|alpha_i| + beta_i) below 1e-4 at some step
    o = lanczos.lanczos_pair(g, int(s[0]), int(t[0]), k_max=60, stop_tol=1e-15)
    k = o["k"]
    ratio = o["beta"][1:k] / np.maximum(np.abs(o["alpha"][:k - 1]) + o["beta"][:k - 1], 1e-300)
    assert ratio.min() < 1e-4, ratio.min()
    G = rd.Graph.from_csr(g)
    for mode in ("fp64", "df64"):
        for onchip in (False, True):
            if mode == "df64" and onchip:
                continue  # double-float vectors: multi-kernel path only
            # the weak edge slows convergence: up to about 500 steps to residual 1e-11
            res = G.query(s, t, mode=mode, k_max=3000, rel_tol=0.0, resid_tol=1e-11, onchip=onchip)
            if mode == "fp64":
                assert np.all(res.status == 0), (mode, onchip, res.status, res.iters)
            else:
                # double-float vectors (about 48 bits) can lose definiteness of I - T_k after such
                # a step: the pair then stops flagged RD_ERR_NUMERIC, never silently
                assert np.all((res.status == 0) | (res.status == rd.RD_ERR_NUMERIC)), res.status
                assert np.any(res.status == 0)
            ok = res.status == 0
            assert rel(res.r[ok], ref[ok]).max() < 1e-8, (mode, onchip, rel(res.r, ref).max())
    for kk in (4, 8, 12, 14):
        orc = np.array([lanczos.lanczos_pair(g, int(a), int(b), k_max=kk)["r"] for a, b in zip(s, t)])
        res = G.query(s, t, mode="fp64", k_max=kk, fixed_k=True, onchip=False)
        m = res.iters == kk
        assert m.any()
        assert rel(res.r[m], orc[m]).max() < 1e-8, (kk, rel(res.r[m], orc[m]).max())


@pytest.mark.parametrize("mode,tol,hist_tol", [("fp64", FP64_TOL, 1e-11), ("fp32", FP32_TOL, 2e-5)])
def test_cluster_whole_recurrence_vs_oracle(rd, mode, tol, hist_tol):
    """Small graphs and few pairs: each pair's whole recurrence runs on a thread-block cluster
    (CTAs holding slices of the vectors, reading each other's through distributed shared
    memory). Against the dense pseudo-inverse or the grid closed form at convergence, the
    oracle's r_k at fixed k, and the one-CTA kernel; a vertex count that no cluster size
    divides, weights, and a heavy row (star centre) included."""
    star = F.star(900)
    cases = [("grid64", W.grid64()[0], np.array([0], np.int32), np.array([4095], np.int32)),
             ("rc1000ln", F.random_connected(1000, 3000, 5, "lognormal"), None, None),
             ("grid37del", F.grid_deleted(37, 0.05, 2), None, None),
             ("star900", star, np.array([3, 10, 0], np.int32), np.array([500, 899, 7], np.int32))]
    for name, g, s, t in cases:
        if s is None:
            s, t = F.random_pairs(g.n, 3, 11)
        ref = (np.array([CF.grid_r(64, 64, 0, 4095)]) if name == "grid64" else dense.DenseRD.of(g).r(s, t))
        G = rd.Graph.from_csr(g)
        kw = dict(mode=mode, k_max=600, rel_tol=0.0, resid_tol=1e-11 if mode == "fp64" else 1e-6)
        res = G.query(s, t, **kw)
        ctas = G.last_stats()["onchip_ctas"]
        assert ctas > 1, (name, ctas)
        assert np.all(res.status == 0), (name, res.status)
        assert rel(res.r, ref).max() < tol, (name, ctas, rel(res.r, ref).max())
        one = G.query(s, t, cluster=False, **kw)
        assert G.last_stats()["onchip_ctas"] == 1
        assert rel(res.r, one.r).max() < tol, name
        k = 12
        orc = [lanczos.lanczos_pair(g, int(a), int(b), k_max=k) for a, b in zip(s, t)]
        fk = G.query(s, t, mode=mode, k_max=k, fixed_k=True)
        assert G.last_stats()["onchip_ctas"] > 1
        # pairs that run all k steps match the oracle's r_k; pairs that break down earlier (the
        # star's Krylov spaces are tiny) hold the exact value, T_i being exact at breakdown
        ko = np.array([o["k"] for o in orc])
        ro = np.array([o["r"] for o in orc])
        m = (fk.iters == k) & (ko == k)
        if m.any():
            assert rel(fk.r[m], ro[m]).max() < hist_tol, (name, rel(fk.r[m], ro[m]).max())
        b = fk.iters < k
        if b.any():
            assert rel(fk.r[b], ref[b]).max() < tol, (name, fk.iters, rel(fk.r[b], ref[b]).max())
        assert m.any() or b.all(), (name, fk.iters, ko)
        assert np.array_equal(G.query(s, t, mode=mode, k_max=k, fixed_k=True).r, fk.r)  # deterministic


def test_scaling_by_four_is_bitwise(rd):
    g = F.grid_deleted(30, 0.05, 5)
    s, t = F.random_pairs(g.n, 8, 3)
    G1 = rd.Graph.from_csr(g)
    G4 = rd.Graph(g.row_ptr, g.col, (4.0 * g.w).astype(np.float32))
    for mode in ["fp64", "fp32"]:
        # the same kernel configuration on both graphs (the autotuner could time them apart)
        r1 = G1.query(s, t, mode=mode, k_max=40, fixed_k=True, tune=False).r
        r4 = G4.query(s, t, mode=mode, k_max=40, fixed_k=True, tune=False).r
        assert np.array_equal(r4 * 4.0, r1)


def test_symmetry_in_s_t(rd):
    g = F.random_connected(200, 400, 12, "lognormal")
    s, t = F.random_pairs(g.n, 16, 5)
    G = rd.Graph.from_csr(g)
    a = G.query(s, t, mode="fp64", rel_tol=0.0, resid_tol=1e-12).r
    b = G.query(t, s, mode="fp64", rel_tol=0.0, resid_tol=1e-12).r
    assert rel(a, b).max() < 1e-10


# grad_w_out is float32 by the ABI, so even the FP64 path is compared at FP32 output precision
@pytest.mark.parametrize("mode,tol", [("fp64", 1e-6), ("fp32", 2e-4)])
def test_edge_grad_vs_dense(rd, mode, tol):
    g = F.random_connected(120, 260, 31, "lognormal")
    s, t = F.random_pairs(g.n, 6, 9)
    gbar = np.linspace(-1.0, 2.0, 6)
    D = dense.DenseRD.of(g)
    ref = D.edge_grad(s, t, gbar)
    G = rd.Graph.from_csr(g)
    gw, r = G.edge_grad(s, t, gbar, mode=mode, k_max=400, rel_tol=0.0,
                        resid_tol=1e-13 if mode == "fp64" else 1e-6)
    assert rel(r, D.r(s, t)).max() < (FP64_TOL if mode == "fp64" else FP32_TOL)
    scale = np.abs(ref).max()
    assert np.abs(gw - ref).max() / scale < tol, np.abs(gw - ref).max() / scale


def test_potential_vs_dense(rd):
    g = F.random_connected(90, 200, 13, "uniform")
    s, t = F.random_pairs(g.n, 4, 6)
    D = dense.DenseRD.of(g)
    G = rd.Graph.from_csr(g)
    phi, r = G.potential(s, t, mode="fp64", rel_tol=0.0, resid_tol=1e-13)
    for p in range(4):
        ref = D.potential(int(s[p]), int(t[p]))
        got = phi[p].astype(np.float64)
        # defined up to a constant: compare edge differences
        rows = g.rows()
        d_ref = ref[rows] - ref[g.col]
        d_got = got[rows] - got[g.col]
        assert np.abs(d_got - d_ref).max() < 1e-6 * np.abs(d_ref).max()


def test_torch_device_io_and_autograd(rd):
    import torch

    g = F.random_connected(100, 220, 19, "uniform")
    s, t = F.random_pairs(g.n, 5, 4)
    G = rd.Graph.from_csr(g)
    sd = torch.from_numpy(s).cuda()
    td = torch.from_numpy(t).cuda()
    res = G.query(sd, td, mode="fp64", rel_tol=0.0, resid_tol=1e-12)
    assert res.r.is_cuda
    ref = dense.DenseRD.of(g).r(s, t)
    assert rel(res.r.cpu().numpy(), ref).max() < FP64_TOL
    w = torch.from_numpy(g.w).cuda().requires_grad_(True)
    opts = dict(mode="fp64", rel_tol=0.0, resid_tol=1e-13)
    r = rd.ResistanceDistance.apply(w, G, sd, td, opts)
    loss = (r * torch.arange(1, 6, device="cuda", dtype=torch.float64)).sum()
    loss.backward()
    refg = dense.DenseRD.of(g).edge_grad(s, t, np.arange(1, 6, dtype=np.float64))
    got = w.grad.cpu().numpy().astype(np.float64)
    assert np.abs(got - refg).max() / np.abs(refg).max() < 1e-6


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_compaction_matches_fixed_layout(rd, mode):
    """Packing converged pairs into narrower blocks changes no pair's result beyond the
    reduction-order rounding of the narrower kernels (which can move a borderline stop
    decision by one step, so both runs are also compared with the oracle)."""
    if mode == "fp64":
        g = F.grid_deleted(60, 0.05, 11)     # distances vary, so pairs stop at different k
        s, t = F.random_pairs(g.n, 200, 13)
        kw = dict(mode=mode, k_max=600, rel_tol=1e-10)
        ref = dense.DenseRD.of(g).r(s, t)
        tol_ab, tol_ref = 1e-8, 1e-8
    else:
        # mean degree 4: the pairs need 10 to 16 steps, so half of them stop while the rest run on
        g, s, t = W.chunglu(20000, 2.1, 4.0, 40000, 200, 31)
        kw = dict(mode=mode, k_max=200, rel_tol=1e-7)
        ref, _, _ = lanczos.lanczos_batch(g, s, t, k_max=200, stop_tol=1e-13, threads=0)
        tol_ab, tol_ref = 2e-6, FP32_TOL
    G = rd.Graph.from_csr(g)
    kw["onchip"] = False
    a = G.query(s, t, **kw)
    st = G.last_stats()
    b = G.query(s, t, compact=False, **kw)
    assert st["compactions"] >= 1 and st["device_loop"] == 1
    assert np.abs(a.iters.astype(int) - b.iters.astype(int)).max() <= 1
    assert rel(a.r, b.r).max() < tol_ab
    assert rel(a.r, ref).max() < tol_ref
    # the host-driven loop packs at the same steps: bitwise the same results
    c = G.query(s, t, device_loop=False, **kw)
    assert np.array_equal(c.r, a.r) and np.array_equal(c.iters, a.iters)
    assert G.last_stats()["compactions"] >= st["compactions"]


@pytest.mark.parametrize("mode", ["fp64", "df64"])
def test_async_kernel_8byte_elements(rd, mode):
    """The async row-stream SpMM with two 8-byte elements per 16-byte lane slot (FP64, or
    double-float as hi/lo pairs): on a weighted power-law graph with heavy rows and on a
    weighted road-like grid, every slab width agrees with the oracle at convergence, with the
    row-group kernel at fixed k, and with itself bitwise on a repeat."""
    cl, s_cl, t_cl = W.chunglu(20000, 2.1, 20.0, 200000, 37, 77, weights="lognormal")
    assert np.diff(cl.row_ptr).max() > 256  # heavy rows present
    gd = F.grid_deleted(48, 0.05, 5)
    gd = F.weighted(gd, F.lognormal_edge_weights(gd.m, 0.0, 0.5, 6))
    s_g, t_g = F.random_pairs(gd.n, 21, 8)
    for g, s, t, k_max in ((cl, s_cl, t_cl, 300), (gd, s_g, t_g, 3000)):
        G = rd.Graph.from_csr(g)
        ref, _, _ = lanczos.lanczos_batch(g, s, t, k_max=k_max, stop_tol=1e-15, threads=0)
        for tile in [16, 32, 64]:
            kw = dict(mode=mode, kernel="async", rhs_tile=tile, compact=False)
            res = G.query(s, t, k_max=k_max, rel_tol=0.0, resid_tol=1e-11, **kw)
            st = G.last_stats()
            assert st["kernel"] == 5 and st["rhs_tile"] == tile
            assert np.all(res.status >= 0)
            assert rel(res.r, ref).max() < FP64_TOL, (tile, rel(res.r, ref).max())
            fa = G.query(s, t, k_max=20, fixed_k=True, **kw)
            fg = G.query(s, t, mode=mode, kernel="group", rhs_tile=tile, compact=False, k_max=20, fixed_k=True)
            assert rel(fa.r, fg.r).max() < 1e-11, (tile, rel(fa.r, fg.r).max())
            assert np.array_equal(G.query(s, t, k_max=20, fixed_k=True, **kw).r, fa.r)
        G.close()


def test_async_kernel_scattered_heavy_rows(rd):
    """The async kernel's row groups take contiguous shares of the tasks and stream each run of
    light rows between heavy rows without a break; the pre-pass streams runs of contiguous
    chunks. On R-MAT, whose heavy rows are scattered among light ones (not the leading ids as
    in Chung-Lu), every tile width agrees with the oracle and with the row-stream kernel."""
    from graphgen.graph import largest_component

    g = largest_component(F.rmat(15, 16, 0.57, 0.19, 0.19, 12))
    d = np.diff(g.row_ptr)
    heavy = np.nonzero(d > 256)[0]
    assert heavy.size > 10 and np.any(np.diff(heavy) > 1)  # heavy rows present, not contiguous
    s, t = F.random_pairs(g.n, 53, 19)
    G = rd.Graph.from_csr(g)
    ref, _, _ = lanczos.lanczos_batch(g, s, t, k_max=300, stop_tol=1e-14, threads=0)
    for tile in [16, 32, 64, 128]:
        kw = dict(mode="fp32", kernel="async", rhs_tile=tile, compact=False)
        res = G.query(s, t, k_max=300, rel_tol=0.0, resid_tol=1e-7, **kw)
        assert G.last_stats()["kernel"] == 5
        assert rel(res.r, ref).max() < FP32_TOL, (tile, rel(res.r, ref).max())
        fa = G.query(s, t, k_max=20, fixed_k=True, **kw)
        fs = G.query(s, t, mode="fp32", kernel="stream", rhs_tile=tile, compact=False, k_max=20, fixed_k=True)
        assert rel(fa.r, fs.r).max() < 2e-6, (tile, rel(fa.r, fs.r).max())


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_flow_kirchhoff_and_dense(rd, mode):
    """Electric flows: f(e) = phi(u) - phi(v) against the dense potential, and Kirchhoff's
    current law: the currents w_e f(e) out of every vertex sum to +1 at s, -1 at t, 0 elsewhere."""
    g = F.random_connected(150, 400, 23, "lognormal")
    s, t = F.random_pairs(g.n, 5, 8)
    G = rd.Graph.from_csr(g)
    f, r = G.flow(s, t, mode=mode, k_max=600, rel_tol=0.0, resid_tol=1e-12 if mode == "fp64" else 1e-6)
    D = dense.DenseRD.of(g)
    rows = g.rows()
    tol = 1e-6 if mode == "fp64" else 1e-4
    for p in range(len(s)):
        phi = D.potential(int(s[p]), int(t[p]))
        ref = phi[rows] - phi[g.col]
        assert np.abs(f[p] - ref).max() < tol * np.abs(ref).max()
        net = np.zeros(g.n)
        np.add.at(net, rows, g.w.astype(np.float64) * f[p].astype(np.float64))
        want = np.zeros(g.n)
        want[s[p]] += 1.0
        want[t[p]] -= 1.0
        assert np.abs(net - want).max() < 10 * tol


def test_power_method_matches_oracle_and_needs_more_steps(rd):
    """Algorithm 1 on the GPU equals the FP64 oracle step by step; on a grid (large
    condition number) it needs many times more steps than the Lanczos iteration to reach
    relative error 1e-6 (the speed-up the paper reports for road networks)."""
    g = F.grid_deleted(30, 0.05, 7)
    s, t = F.random_pairs(g.n, 4, 9)
    G = rd.Graph.from_csr(g)
    steps = 20000
    r, hist = G.power_method(s, t, steps, mode="fp64", history=True)
    for p in range(2):
        ref = power.power_method(g, int(s[p]), int(t[p]), steps)
        assert np.abs(hist[:, p] - ref).max() < 1e-12 * np.abs(ref).max() + 1e-14
    exact = dense.DenseRD.of(g).r(s, t)
    lz = G.query(s, t, mode="fp64", k_max=2000, rel_tol=0.0, resid_tol=1e-12)
    k_lz = np.array([np.argmax(np.abs(lanczos.lanczos_pair(g, int(a), int(b), 300)["r_hist"] / e - 1) <= 1e-6) + 1
                     for a, b, e in zip(s, t, exact)])
    rel_pm = np.abs(hist / exact[None, :] - 1)
    k_pm = np.array([np.argmax(rel_pm[:, p] <= 1e-6) for p in range(len(s))])
    assert np.all(rel_pm[-1] <= 1e-6)
    assert np.all(k_pm > 5 * k_lz), (k_pm, k_lz)
    assert rel(lz.r, exact).max() < 1e-9


def test_triangle_weights_then_weighted_query(rd):
    """Triangle-count weights (the weighted setting of the paper's experiments): each stored
    entry gets the number of triangles through its edge (1 if none), as (A A) o A counts
    them; the weighted query then matches the dense oracle on those weights."""
    import scipy.sparse as sp

    g, s, t = W.chunglu(5000, 2.1, 20.0, 50000, 8, 5)
    G = rd.Graph.from_csr(g)
    w = G.triangle_weights()
    A = sp.csr_matrix((np.ones(g.nnz), g.col, g.row_ptr), shape=(g.n, g.n))
    tri = (A @ A).multiply(A).tocsr()
    tri.sort_indices()
    ref = np.asarray(tri[g.rows(), g.col]).ravel()
    ref = np.where(ref > 0, ref, 1.0)
    assert np.array_equal(w, ref.astype(np.float32))
    k = F.complete(6)
    assert np.all(rd.Graph.from_csr(k).triangle_weights() == 4.0)      # K_6: n - 2 triangles per edge
    gw = g.with_weights(w)
    G.set_weights(w)
    res = G.query(s, t, mode="fp64", rel_tol=0.0, resid_tol=1e-12)
    assert rel(res.r, dense.DenseRD.of(gw).r(s, t)).max() < FP64_TOL


@pytest.mark.parametrize("family", ["er", "ba"])
def test_er_ba_workloads_vs_dense(rd, family):
    """Erdos-Renyi and Barabasi-Albert graphs (the scalability and density experiments):
    converged queries against the dense oracle, fixed k = 20 against the oracle's rhat_20."""
    import math

    n = 1500
    g = F.erdos_renyi(n, int(n * math.log(n)), 4) if family == "er" else F.barabasi_albert(n, 7, 4)
    s, t = F.random_pairs(g.n, 20, 6)
    G = rd.Graph.from_csr(g)
    ref = dense.DenseRD.of(g).r(s, t)
    for mode, tol in [("fp64", FP64_TOL), ("fp32", FP32_TOL)]:
        res = G.query(s, t, mode=mode, rel_tol=0.0, resid_tol=1e-12 if mode == "fp64" else 1e-6)
        assert rel(res.r, ref).max() < tol
    r20 = G.query(s, t, mode="fp64", k_max=20, fixed_k=True).r
    for p in range(3):
        assert rel([r20[p]], [lanczos.lanczos_pair(g, int(s[p]), int(t[p]), 20)["r"]])[0] < 1e-11


def test_plain_kernels_agree(rd):
    """The single-pair path: warp-per-task SpMV, row-group and row-stream kernels agree."""
    g, s, t = W.chunglu(30000, 2.1, 20.0, 300000, 6, 17)
    G = rd.Graph.from_csr(g)
    out = [G.query(s, t, mode=m, k_max=40, fixed_k=True, plain=True, kernel=k).r
           for m in ["fp64"] for k in ["tuned", "group", "stream", "group_sorted"]]
    assert G.last_stats()["kernel"] == 3 and G.last_stats()["row_order"] == 1
    assert max(rel(o, out[0]).max() for o in out[1:]) < 1e-12
    r32 = G.query(s, t, mode="fp32", k_max=40, fixed_k=True, plain=True).r
    assert rel(r32, out[0]).max() < 2e-5


@pytest.mark.parametrize("mode,tol", [("fp64", 1e-11), ("fp32", 2e-6)])
def test_onchip_path_matches_multikernel_path(rd, mode, tol):
    """Small graphs run as one whole-recurrence kernel (one block per pair); the result equals
    the multi-kernel path's within reduction-order rounding, for plain and weighted graphs with
    heavy rows (a star hub) and tolerance stops."""
    a = F.random_connected(3000, 9000, 41, "lognormal")
    hub = F.star(400)
    ea, eb, wa = a.undirected_edges()
    ha, hb, _ = hub.undirected_edges()
    g = to_csr(3000, np.concatenate([ea, ha]), np.concatenate([eb, hb]),
               np.concatenate([wa, np.ones(ha.size, np.float32)]))
    s, t = F.random_pairs(g.n, 33, 4)
    G = rd.Graph.from_csr(g)
    for kw in [dict(k_max=30, fixed_k=True), dict(k_max=400, rel_tol=1e-9 if mode == "fp64" else 1e-6)]:
        on = G.query(s, t, mode=mode, **kw)
        off = G.query(s, t, mode=mode, onchip=False, **kw)
        assert np.abs(on.iters.astype(int) - off.iters.astype(int)).max() <= 1
        assert rel(on.r, off.r).max() < (tol if "fixed_k" in kw else 50 * tol)
    ref = dense.DenseRD.of(g).r(s, t)
    res = G.query(s, t, mode=mode, rel_tol=0.0, resid_tol=1e-12 if mode == "fp64" else 1e-6)
    assert rel(res.r, ref).max() < (FP64_TOL if mode == "fp64" else FP32_TOL)


def test_workspace_allocation_failure_is_reported(rd):
    """A request whose workspace cannot be allocated returns RD_ERR_OOM and leaves the graph
    usable (allocation failure is the one device fault the library injects on purpose)."""
    g = F.path(200000)
    G = rd.Graph.from_csr(g)
    s1, t1 = np.array([0, 5], np.int32), np.array([7, 99], np.int32)
    before = G.query(s1, t1, mode="fp64", k_max=50, fixed_k=True).r
    big = 1 << 22                      # 4M pairs x 200k rows x 2 blocks x 4 bytes: ~6.4 TB
    s = np.zeros(big, np.int32)
    t = np.ones(big, np.int32)
    with pytest.raises(rd.RDError) as e:
        G.query(s, t, mode="fp32", k_max=4)
    assert e.value.status == rd.RD_ERR_OOM
    after = G.query(s1, t1, mode="fp64", k_max=50, fixed_k=True).r
    assert np.array_equal(before, after)


@pytest.mark.parametrize("mode,tol", [("fp64", FP64_TOL), ("fp32", FP32_TOL)])
def test_autotuner_choice_is_used_and_correct(rd, mode, tol):
    """rd_autotune times the candidates on this graph and keeps the fastest; later queries use
    it (stats say so), agree with the oracle, and with the fixed-rule configuration."""
    g, s, t = W.chunglu(30000, 2.1, 20.0, 300000, 48, 91)
    G = rd.Graph.from_csr(g)
    ref, _, _ = lanczos.lanczos_batch(g, s, t, k_max=200, stop_tol=1e-14, threads=0)
    pick = G.autotune(len(s), mode=mode)
    assert pick["kernel"] in ((1, 2, 3) if mode == "fp64" else (1, 2, 3, 5)) and pick["rhs_tile"] >= 8
    res = G.query(s, t, mode=mode, k_max=200, rel_tol=0.0, resid_tol=1e-12 if mode == "fp64" else 1e-7,
                  compact=False)
    st = G.last_stats()
    assert st["tuned"] == 1 and st["rhs_tile"] == pick["rhs_tile"] and st["kernel"] == pick["kernel"]
    assert rel(res.r, ref).max() < tol
    fixed = G.query(s, t, mode=mode, k_max=200, rel_tol=0.0, resid_tol=1e-12 if mode == "fp64" else 1e-7,
                    compact=False, tune=False)
    assert G.last_stats()["tuned"] == 0
    assert rel(fixed.r, ref).max() < tol
    # the single-column path is tuned separately
    one = G.autotune(1, mode=mode, plain=True)
    assert one["rhs_tile"] == 1 and one["kernel"] in (1, 2, 3, 4)
    p = G.query(s[:3], t[:3], mode=mode, plain=True, k_max=200, rel_tol=0.0,
                resid_tol=1e-12 if mode == "fp64" else 1e-7)
    assert G.last_stats()["kernel"] == one["kernel"]
    assert rel(p.r, ref[:3]).max() < tol


def test_autotuner_first_use_and_arguments(rd):
    """A query with default options tunes its width classes on first use (compacting query:
    down to the narrowest tile); explicit tiles bypass the table; bad calls are rejected."""
    g, s, t = W.chunglu(20000, 2.1, 20.0, 200000, 100, 5)
    G = rd.Graph.from_csr(g)
    a = G.query(s, t, k_max=200, rel_tol=1e-6)
    assert G.last_stats()["tuned"] == 1
    b = G.query(s, t, k_max=200, rel_tol=1e-6)
    assert np.array_equal(a.r, b.r)              # same table entry, same summation order
    G.query(s, t, k_max=200, rel_tol=1e-6, rhs_tile=32)
    assert G.last_stats()["tuned"] == 0 and G.last_stats()["rhs_tile"] == 32
    with pytest.raises(rd.RDError) as e:
        G.autotune(16, rhs_tile=16)
    assert e.value.status == rd.RD_ERR_INVALID_ARG
    with pytest.raises(rd.RDError) as e:
        G.autotune(0)
    assert e.value.status == rd.RD_ERR_INVALID_ARG


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_graph_replay_is_bitwise_the_launch_loop(rd, mode):
    """Steps replayed from the captured one-step CUDA graph (step index in device memory),
    and the device-resident loop (a conditional while node repeating the step until every
    pair stops or a column compaction is due), give bitwise the results of launching every
    kernel from the host: compacting query with the error-estimate stop, fixed k, a k_max
    reached with pairs still active, the plain path, and the gradient (potential built
    during the forward steps, or by the replay pass, which must regenerate the forward
    vectors)."""
    g, s, t = W.chunglu(20000, 2.1, 20.0, 200000, 70, 13)
    G = rd.Graph.from_csr(g)
    for kw in (dict(k_max=5, rel_tol=1e-12), dict(k_max=200, rel_tol=1e-7),
               dict(k_max=200, rel_tol=0.0, resid_tol=1e-9), dict(k_max=7, fixed_k=True),
               dict(k_max=200, rel_tol=1e-7, compact=False)):
        a = G.query(s, t, mode=mode, **kw)
        ga = G.last_stats()
        assert ga["device_loop"] == 1 and ga["steps"] <= kw["k_max"], kw
        b = G.query(s, t, mode=mode, graph=False, **kw)
        gb = G.last_stats()
        assert gb["device_loop"] == 0
        assert np.array_equal(a.r, b.r), kw
        assert np.array_equal(a.iters, b.iters) and np.array_equal(a.status, b.status), kw
        # the device loop tests the current count before packing, so it skips a packing after
        # the last pair stopped that the lagged host poll still makes
        assert ga["compactions"] <= gb["compactions"], kw
        c = G.query(s, t, mode=mode, device_loop=False, **kw)  # one-step graph, host-driven
        assert G.last_stats()["device_loop"] == 0
        assert np.array_equal(c.r, b.r) and np.array_equal(c.iters, b.iters), kw
        assert G.last_stats()["compactions"] == gb["compactions"], kw
    pa = G.query(s[:5], t[:5], mode=mode, plain=True, k_max=200, rel_tol=1e-7)
    pb = G.query(s[:5], t[:5], mode=mode, plain=True, k_max=200, rel_tol=1e-7, graph=False)
    assert np.array_equal(pa.r, pb.r) and np.array_equal(pa.iters, pb.iters)
    ga, ra = G.edge_grad(s[:16], t[:16], None, mode=mode, k_max=200, rel_tol=0.0, resid_tol=1e-9)
    gb, rb = G.edge_grad(s[:16], t[:16], None, mode=mode, k_max=200, rel_tol=0.0, resid_tol=1e-9, graph=False)
    assert np.array_equal(ra, rb) and np.array_equal(ga, gb)
    kw = dict(mode=mode, k_max=200, rel_tol=0.0, resid_tol=1e-9, potential_mode="replay")
    ga, ra = G.edge_grad(s[:16], t[:16], None, **kw)
    gb, rb = G.edge_grad(s[:16], t[:16], None, graph=False, **kw)
    assert np.array_equal(ra, rb) and np.array_equal(ga, gb)
    ref, _, _ = lanczos.lanczos_batch(g, s, t, k_max=200, stop_tol=1e-14, threads=0)
    assert rel(a.r, ref).max() < 1e-7        # the last query's rel_tol


@pytest.mark.parametrize("family", ["chunglu", "rmat", "ba", "grid_del", "grid"])
def test_error_estimate_stop_meets_rel_tol(rd, family):
    """The rel_tol stop (geometric tail estimate) returns estimates within rel_tol of the
    converged value on the method's workload families, and on fast-mixing graphs stops no
    later than the delayed-sum estimate."""
    from graphgen.graph import largest_component

    if family == "chunglu":
        g, s, t = W.chunglu(30000, 2.1, 20.0, 300000, 32, 41)
    elif family == "rmat":
        g = largest_component(F.rmat(14, 16, 0.57, 0.19, 0.19, 8))
        s, t = F.random_pairs(g.n, 32, 6)
    elif family == "ba":
        g = F.barabasi_albert(8000, 4, 6)
        s, t = F.random_pairs(g.n, 32, 7)
    elif family == "grid_del":
        g = F.grid_deleted(40, 0.05, 11)
        s, t = F.random_pairs(g.n, 16, 8)
    else:
        g = F.grid(48)
        s, t = F.random_pairs(g.n, 16, 9)
    ref, _, _ = lanczos.lanczos_batch(g, s, t, k_max=5000, stop_tol=1e-15, threads=0)
    G = rd.Graph.from_csr(g)
    for tol in (1e-4, 1e-6, 1e-8):
        res = G.query(s, t, mode="fp64", k_max=5000, rel_tol=tol)
        assert np.all(res.status == 0)
        assert rel(res.r, ref).max() <= tol, (family, tol, rel(res.r, ref).max())
        if family in ("chunglu", "rmat", "ba"):
            old = G.query(s, t, mode="fp64", k_max=5000, rel_tol=tol, estimate="delayed")
            assert np.all(res.iters <= old.iters)


@pytest.mark.parametrize("kernel", ["tuned", "group", "stream", "tasks"])
def test_double_float_mode_vs_oracle(rd, kernel):
    """RD_MODE_DF64 (vectors as FP32 pairs, FP64-class accuracy on the FP32 units): fixed-k
    estimates equal the FP64 oracle's, converged values equal the dense pseudo-inverse, on
    unweighted and weighted graphs, batched (with compaction and graph replay) and plain."""
    for g in (F.grid_deleted(24, 0.05, 9), F.random_connected(300, 900, 31, "lognormal")):
        s, t = F.random_pairs(g.n, 9, 2)
        G = rd.Graph.from_csr(g)
        plain = kernel == "tasks"
        kw = dict(kernel=kernel, onchip=False, plain=plain)
        for k in (1, 3, 17, 40):
            ref = np.array([lanczos.lanczos_pair(g, int(a), int(b), k_max=k)["r"] for a, b in zip(s, t)])
            res = G.query(s, t, mode="df64", k_max=k, fixed_k=True, **kw)
            assert rel(res.r, ref).max() < 1e-11, (k, rel(res.r, ref).max())
        exact = dense.DenseRD.of(g).r(s, t)
        res = G.query(s, t, mode="df64", k_max=2000, rel_tol=0.0, resid_tol=1e-12, **kw)
        assert np.all(res.status == 0)
        assert rel(res.r, exact).max() < FP64_TOL
        if not plain:
            gb = G.query(s, t, mode="df64", k_max=2000, rel_tol=0.0, resid_tol=1e-12, graph=False, **kw)
            assert np.array_equal(gb.r, res.r)


def test_double_float_mode_batched_chunglu(rd):
    """Batched double-float query with the error-estimate stop, compaction and the tuned
    kernels on a power-law graph: within 1e-9 of the oracle; the other entry points run the
    mode as FP64."""
    # mean degree 4: the pairs need 21 to 27 steps, so most stop while the rest run on packed
    g, s, t = W.chunglu(30000, 2.1, 4.0, 60000, 100, 23)
    G = rd.Graph.from_csr(g)
    ref, _, _ = lanczos.lanczos_batch(g, s, t, k_max=300, stop_tol=1e-15, threads=0)
    res = G.query(s, t, mode="df64", k_max=300, rel_tol=0.0, resid_tol=1e-11)
    st = G.last_stats()
    assert st["compactions"] >= 1 and st["device_loop"] == 1
    assert rel(res.r, ref).max() < FP64_TOL
    # the device loop packs with the fused normalise pass (8-byte elements): bitwise the
    # normalise pass followed by the separate packing of the host-driven loop
    hl = G.query(s, t, mode="df64", k_max=300, rel_tol=0.0, resid_tol=1e-11, device_loop=False)
    assert np.array_equal(hl.r, res.r) and np.array_equal(hl.iters, res.iters)
    r64 = G.query(s, t, mode="fp64", k_max=300, rel_tol=0.0, resid_tol=1e-11).r
    assert rel(res.r, r64).max() < 1e-10
    gd, rd_ = G.edge_grad(s[:4], t[:4], None, mode="df64", k_max=300, rel_tol=0.0, resid_tol=1e-11)
    g6, r6 = G.edge_grad(s[:4], t[:4], None, mode="fp64", k_max=300, rel_tol=0.0, resid_tol=1e-11)
    assert np.array_equal(gd, g6) and np.array_equal(rd_, r6)


@pytest.mark.parametrize("mode,tol", [("fp64", 1e-11), ("df64", 1e-11), ("fp32", 2e-5)])
def test_sparse_first_step_matches_dense_first_step(rd, mode, tol):
    """The first step computed from the sparse start vector (only the rows adjacent to s and
    t) agrees with the SpMM over every row: fixed-k estimates and gradients, converged values
    against the dense pseudo-inverse; on a power-law graph with hub endpoints (hub-hub pairs
    share many neighbours), a grid with adjacent pairs and pairs whose endpoints share one or
    two neighbours, and a weighted graph. Rows not sorted by column, or weights not symmetric
    bit for bit, take the SpMM."""
    cl, s_cl, t_cl = W.chunglu(20000, 2.1, 20.0, 200000, 24, 77)
    hubs = np.argsort(np.diff(cl.row_ptr))[-3:].astype(np.int32)
    s_cl = np.concatenate([s_cl, hubs, hubs[2:], t_cl[:1]]).astype(np.int32)
    t_cl = np.concatenate([t_cl, np.roll(hubs, 1), s_cl[:1], hubs[:1]]).astype(np.int32)
    grid = F.grid(20)
    s_g = np.array([0, 21, 21, 0, 105, 399, 7], np.int32)
    t_g = np.array([1, 42, 23, 399, 106, 398, 7], np.int32)
    wg = F.random_connected(300, 900, 31, "lognormal")
    s_w, t_w = F.random_pairs(wg.n, 12, 4)
    for g, s, t in ((cl, s_cl, t_cl), (grid, s_g, t_g), (wg, s_w, t_w)):
        G = rd.Graph.from_csr(g)
        kw = dict(mode=mode, k_max=9, fixed_k=True, onchip=False)
        a = G.query(s, t, **kw)
        assert G.last_stats()["sparse_first"] == 1
        b = G.query(s, t, sparse_first=False, **kw)
        assert G.last_stats()["sparse_first"] == 0
        nz = s != t
        assert np.all(a.r[~nz] == 0.0) and np.array_equal(a.status, b.status)
        assert rel(a.r[nz], b.r[nz]).max() < tol, (g.name, rel(a.r[nz], b.r[nz]).max())
        ref = np.array([lanczos.lanczos_pair(g, int(x), int(y), k_max=9)["r"] if x != y else 0.0
                        for x, y in zip(s, t)])
        assert rel(a.r[nz], ref[nz]).max() < tol
        conv = G.query(s, t, mode=mode, k_max=3000, rel_tol=0.0, resid_tol=1e-12 if mode != "fp32" else 1e-6)
        assert np.all(conv.status == 0)
        if g.n <= 400 or g is wg:
            exact = dense.DenseRD.of(g).r(s[nz], t[nz])
            assert rel(conv.r[nz], exact).max() < (FP64_TOL if mode != "fp32" else FP32_TOL)
        if mode != "df64":
            gk = dict(mode=mode, k_max=12, fixed_k=True)
            ga, ra = G.edge_grad(s[nz][:8], t[nz][:8], None, **gk)
            gb, rb = G.edge_grad(s[nz][:8], t[nz][:8], None, sparse_first=False, **gk)
            assert rel(ra, rb).max() < tol
            assert np.abs(ga - gb).max() <= 50 * tol * np.abs(gb).max()
    # rows in decreasing column order
    col = grid.col.copy()
    for u in range(grid.n):
        col[grid.row_ptr[u]:grid.row_ptr[u + 1]] = col[grid.row_ptr[u]:grid.row_ptr[u + 1]][::-1]
    G2 = rd.Graph(grid.row_ptr, col, None)
    r2 = G2.query(s_g, t_g, mode="fp64", k_max=3000, rel_tol=0.0, resid_tol=1e-12, onchip=False)
    assert G2.last_stats()["sparse_first"] == 0
    nz = s_g != t_g
    assert rel(r2.r[nz], dense.DenseRD.of(grid).r(s_g[nz], t_g[nz])).max() < FP64_TOL
    # one weight of one direction moved by one ulp
    w = wg.w.copy()
    w[0] = np.nextafter(w[0], np.float32(np.inf))
    G3 = rd.Graph(wg.row_ptr, wg.col, w)
    G3.query(s_w, t_w, mode="fp64", k_max=20, fixed_k=True, onchip=False)
    assert G3.last_stats()["sparse_first"] == 0
    G3.set_weights(wg.w)
    G3.query(s_w, t_w, mode="fp64", k_max=20, fixed_k=True, onchip=False)
    assert G3.last_stats()["sparse_first"] == 1


@pytest.mark.parametrize("mode,tol", [("fp64", 1e-9), ("fp32", 3e-4)])
def test_direct_potential_matches_replay_pass(rd, mode, tol):
    """The potential accumulated during the forward steps (p_i = q_i + lambda_i p_{i-1},
    x += mu_i p_i from the LDL^T factors of I - T_i) equals the replay pass's sum of
    ||b|| z_j q_j: gradients, potentials and flows, at fixed k and converged (pairs stopping
    at different steps), on a weighted power-law graph and on a grid; the direct form needs
    one SpMM step per Lanczos step instead of two."""
    cl, s_cl, t_cl = W.chunglu(20000, 2.1, 20.0, 200000, 24, 5, weights="lognormal")
    gd = F.grid_deleted(40, 0.05, 3)
    s_g, t_g = F.random_pairs(gd.n, 12, 4)
    for g, s, t in ((cl, s_cl, t_cl), (gd, s_g, t_g)):
        G = rd.Graph.from_csr(g)
        for kw in (dict(k_max=11, fixed_k=True),
                   dict(k_max=3000, rel_tol=0.0, resid_tol=1e-10 if mode == "fp64" else 1e-6)):
            ga, ra = G.edge_grad(s, t, None, mode=mode, **kw)
            steps_direct = G.last_stats()["spmm_launches"]
            gb, rb = G.edge_grad(s, t, None, mode=mode, potential_mode="replay", **kw)
            assert np.array_equal(ra, rb)                   # the same forward pass
            assert G.last_stats()["spmm_launches"] > steps_direct
            assert np.abs(ga - gb).max() <= tol * np.abs(gb).max(), (g.name, kw, np.abs(ga - gb).max())
            pa, _ = G.potential(s[:6], t[:6], mode=mode, **kw)
            pb, _ = G.potential(s[:6], t[:6], mode=mode, potential_mode="replay", **kw)
            assert np.abs(pa - pb).max() <= tol * np.abs(pb).max()
            fa, _ = G.flow(s[:6], t[:6], mode=mode, **kw)
            fb, _ = G.flow(s[:6], t[:6], mode=mode, potential_mode="replay", **kw)
            assert np.abs(fa - fb).max() <= tol * np.abs(fb).max()
