"""rd_query_noalloc, the query entry point for callers that cannot allocate device memory
(for example code running under another framework's allocator, or a process that reserves
all device memory up front). Its scratch is a fixed array inside the library, so it must
give the same answers as rd_query while leaving the device's free memory untouched.

This file is named so that pytest collects it last: if it fails, a run that stops at
the first failure has already run every other test.
"""
import numpy as np
import pytest

from graphgen import families as F
from graphgen import workloads as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9
FP32_TOL = 1e-5


def _dev(rd, g, s, t):
    import torch

    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    w = None if g.w is None else torch.from_numpy(g.w).cuda()
    return rp, col, w, torch.from_numpy(s).cuda(), torch.from_numpy(t).cuda()


@pytest.mark.parametrize("mode,tol", [("fp32", FP32_TOL), ("fp64", FP64_TOL)])
def test_noalloc_matches_rd_query_on_two_calls(mode, tol):
    import torch

    import paper_2601_11159_gb300 as rd

    g, s, t = W.chunglu(20000, 2.1, 20.0, 200000, 24, 5)
    gw = F.random_connected(3000, 9000, 8, "lognormal")
    sw, tw = F.random_pairs(gw.n, 10, 3)
    for graph, ss, tt in [(g, s, t), (gw, sw, tw)]:
        G = rd.Graph.from_csr(graph)
        kw = dict(mode=mode, k_max=200, rel_tol=0.0, resid_tol=1e-10 if mode == "fp64" else 1e-6)
        ref = G.query(ss, tt, **kw)
        rp, col, w, sd, td = _dev(rd, graph, ss, tt)
        r_out = torch.empty(len(ss), dtype=torch.float64, device="cuda")
        it_out = torch.empty(len(ss), dtype=torch.int32, device="cuda")
        rd.query_noalloc(rp, col, w, sd, td, out=(r_out, it_out), **kw)  # first call: scratch set-up
        torch.cuda.synchronize()
        for call in range(2):
            free_before = torch.cuda.mem_get_info()[0]
            r, it = rd.query_noalloc(rp, col, w, sd, td, out=(r_out, it_out), **kw)
            torch.cuda.synchronize()
            free_after = torch.cuda.mem_get_info()[0]
            assert free_after == free_before, f"call {call} changed free device memory"
            got = r.cpu().numpy()
            rel = np.abs(got - ref.r) / np.abs(ref.r)
            assert rel.max() < tol, (mode, call, rel.max())
        G.close()


@pytest.mark.parametrize("case", ["plain", "onchip"])
def test_noalloc_plain_and_onchip_paths_vs_oracle(case):
    """The per-pair loop (plain=True) and the whole-recurrence kernel that small graphs take
    carve their workspace from the fixed scratch with other widths than the batched path:
    both agree with the CPU oracle and with rd_query, and leave free device memory as it was."""
    import torch

    import paper_2601_11159_gb300 as rd
    from oracle import lanczos

    if case == "plain":
        g = F.random_connected(2000, 5000, 21, "lognormal")
        s, t = F.random_pairs(g.n, 5, 4)
        # onchip=False: the per-pair SpMV loop, not the whole-recurrence kernel this size allows
        kw = dict(mode="fp64", k_max=400, rel_tol=0.0, resid_tol=1e-12, plain=True, onchip=False)
    else:
        g = F.cycle(64)  # three vectors of 64 rows fit in shared memory: one block per pair
        s = np.array([0, 3, 10, 63], np.int32)
        t = np.array([32, 40, 11, 1], np.int32)
        kw = dict(mode="fp64", k_max=200, rel_tol=0.0, resid_tol=1e-12)
    ref = np.array([lanczos.lanczos_pair(g, int(a), int(b), k_max=kw["k_max"], stop_tol=1e-15)["r"]
                    for a, b in zip(s, t)])
    G = rd.Graph.from_csr(g)
    via_graph = G.query(s, t, **kw).r
    rp, col, w, sd, td = _dev(rd, g, s, t)
    r_out = torch.empty(len(s), dtype=torch.float64, device="cuda")
    it_out = torch.empty(len(s), dtype=torch.int32, device="cuda")
    rd.query_noalloc(rp, col, w, sd, td, out=(r_out, it_out), **kw)
    torch.cuda.synchronize()
    for call in range(2):
        free_before = torch.cuda.mem_get_info()[0]
        r, _ = rd.query_noalloc(rp, col, w, sd, td, out=(r_out, it_out), **kw)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before, f"call {call} changed free device memory"
        got = r.cpu().numpy()
        assert (np.abs(got - ref) / ref).max() < FP64_TOL, (case, call)
        assert (np.abs(got - via_graph) / via_graph).max() < FP64_TOL
    if case == "onchip":
        k = np.array([min(abs(int(a) - int(b)), 64 - abs(int(a) - int(b))) for a, b in zip(s, t)])
        assert np.allclose(got, k * (64 - k) / 64.0, rtol=1e-9)  # cycle closed form h(n-h)/n
    G.close()


def test_noalloc_rejects_tensors_it_would_have_to_convert():
    """The Python entry point passes tensors to the C call as they are: a dtype, layout or
    size that would need a converted copy (a device allocation) is refused up front."""
    import torch

    import paper_2601_11159_gb300 as rd

    g = F.cycle(10)
    rp, col, w, sd, td = _dev(rd, g, np.array([0, 1], np.int32), np.array([5, 6], np.int32))
    r_ok = torch.empty(2, dtype=torch.float64, device="cuda")
    it_ok = torch.empty(2, dtype=torch.int32, device="cuda")
    with pytest.raises(TypeError):
        rd.query_noalloc(rp, col.to(torch.int64), None, sd, td)       # int64 column ids
    with pytest.raises(TypeError):
        rd.query_noalloc(rp.to(torch.int32), col, None, sd, td)       # int32 row_ptr
    s2 = torch.stack([sd, sd], 1)[:, 0]                               # non-contiguous view
    assert not s2.is_contiguous()
    with pytest.raises(TypeError):
        rd.query_noalloc(rp, col, None, s2, td)
    with pytest.raises(ValueError):
        rd.query_noalloc(rp, col, None, sd, td[:1])                   # t shorter than s
    with pytest.raises(TypeError):
        rd.query_noalloc(rp, col, None, sd, td, out=(r_ok.float(), it_ok))   # float32 r
    with pytest.raises(ValueError):
        rd.query_noalloc(rp, col, None, sd, td, out=(r_ok[:1], it_ok))       # too short
    with pytest.raises(TypeError):
        rd.query_noalloc(rp, col, None, sd, td, out=(r_ok, it_ok.to(torch.int64)))
    r, it = rd.query_noalloc(rp, col, None, sd, td, out=(r_ok, it_ok), mode="fp64", rel_tol=0.0,
                             resid_tol=1e-12)
    assert np.allclose(r.cpu().numpy(), [2.5, 2.5], rtol=1e-9)


def test_noalloc_rejects_oversized_requests_and_host_pointers():
    import torch

    import paper_2601_11159_gb300 as rd

    big = F.path(3_000_000)  # 24 bytes of degrees per vertex alone exceed the fixed scratch
    rp, col, w, sd, td = _dev(rd, big, np.array([0], np.int32), np.array([5], np.int32))
    with pytest.raises(rd.RDError) as e:
        rd.query_noalloc(rp, col, None, sd, td)
    assert e.value.status == rd.RD_ERR_INVALID_ARG and "scratch" in str(e.value)
    small = F.cycle(10)
    rp, col, w, sd, td = _dev(rd, small, np.array([0], np.int32), np.array([5], np.int32))
    with pytest.raises(TypeError):
        rd.query_noalloc(rp.cpu(), col, None, sd, td)
    r, it = rd.query_noalloc(rp, col, None, sd, td, mode="fp64", rel_tol=0.0, resid_tol=1e-12)
    assert float(r.cpu()[0]) == pytest.approx(5 * 5 / 10, rel=1e-9)
