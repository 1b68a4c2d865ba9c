"""The C-ABI library builds, loads and exports every symbol its header declares;
argument validation that needs no GPU. CPU only."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2601_11159_gb300 import build, _lib

    build.build()
    return _lib.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rd_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["rd_graph_create", "rd_graph_destroy", "rd_query", "rd_edge_grad", "rd_status_string"]:
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/rd.h but not exported"
    from paper_2601_11159_gb300 import _lib

    assert sorted(_lib.EXPORTS) == declared_functions()


def test_status_strings_and_defaults(lib):
    from paper_2601_11159_gb300 import _lib

    for code in [0, 1, -1, -2, -3, -4, -5, -6, -7, -8]:
        assert lib.rd_status_string(code)
    o = _lib.QueryOpts()
    lib.rd_query_opts_init(C.byref(o))
    assert o.k_max == 1000 and o.mode == _lib.RD_MODE_FP32V_FP64S and o.rel_tol == pytest.approx(1e-7)


def test_invalid_arguments_rejected_before_device_work(lib):
    from paper_2601_11159_gb300 import _lib

    h = C.c_void_p()
    rp = (C.c_int64 * 2)(0, 0)
    assert lib.rd_graph_create(C.byref(h), 0, 0, rp, None, None, 0, None) == _lib.RD_ERR_INVALID_ARG
    assert h.value is None
    assert lib.rd_graph_create(None, 1, 0, rp, None, None, 0, None) == _lib.RD_ERR_INVALID_ARG
    assert lib.rd_graph_create(C.byref(h), 3, -1, rp, None, None, 0, None) == _lib.RD_ERR_INVALID_ARG
    assert lib.rd_query(None, None, None, 1, None, None, None, None, None, None) == _lib.RD_ERR_INVALID_ARG
    assert b"NULL" in lib.rd_last_error()
    assert lib.rd_graph_destroy(None) == _lib.RD_OK


def test_package_has_no_cpu_fallback(monkeypatch, tmp_path):
    """The binding raises when the library is missing instead of computing anything itself."""
    from paper_2601_11159_gb300 import _lib

    with pytest.raises(ImportError):
        _lib.load(str(tmp_path / "missing.so"))
    pkg = os.path.join(ROOT, "paper_2601_11159_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt


def _header_struct_fields(name):
    """(type, field) pairs of `typedef struct { ... } name;` in include/rd.h, in order."""
    import re

    text = open(os.path.join(ROOT, "include", "rd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    end = re.search(r"\}\s*" + name + r"\s*;", text)
    assert end, name
    start = text.rfind("typedef struct", 0, end.start())
    body = text[text.index("{", start) + 1:end.start()]
    out = []
    for decl in body.split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        typ, *names = decl.replace(",", " ").split()
        out.extend((typ, n) for n in names)
    return out


@pytest.mark.parametrize("cname,pyname", [("rd_query_opts", "QueryOpts"), ("rd_call_stats", "CallStats")])
def test_ctypes_structs_match_header(cname, pyname):
    """The binding's ctypes mirrors of the ABI structs have the header's fields, order and types."""
    from paper_2601_11159_gb300 import _lib

    ctype = {"int32_t": C.c_int32, "int64_t": C.c_int64, "double": C.c_double, "uint32_t": C.c_uint32}
    hdr = _header_struct_fields(cname)
    py = getattr(_lib, pyname)._fields_
    assert [n for _, n in hdr] == [n for n, _ in py]
    for (t, n), (_, pt) in zip(hdr, py):
        assert ctype[t] == pt, (cname, n, t, pt)


def test_header_constants_match_the_binding():
    """Every #define RD_* value in the header equals the binding's constant of that name, and
    the binding's keyword options set exactly the documented flags."""
    from paper_2601_11159_gb300 import _lib

    src = open(os.path.join(ROOT, "include", "rd.h")).read()
    defines = dict(re.findall(r"#define\s+(RD_[A-Z0-9_]+)\s+(\d+)u?", src))
    assert defines
    for name, value in defines.items():
        assert getattr(_lib, name) == int(value), name
    import paper_2601_11159_gb300 as rd

    base = rd._opts().flags
    assert base == 0
    assert rd._opts(sparse_first=False).flags == _lib.RD_Q_DENSE_FIRST
    assert rd._opts(potential_mode="replay").flags == _lib.RD_Q_REPLAY_POTENTIAL
    assert rd._opts(graph=False, tune=False).flags == _lib.RD_Q_NO_GRAPH | _lib.RD_Q_NO_TUNE
    assert rd._opts(estimate="delayed").flags == _lib.RD_Q_EST_DELAYED
    assert rd._opts(cluster=False).flags == _lib.RD_Q_NO_CLUSTER
    assert rd._opts(device_loop=False).flags == _lib.RD_Q_NO_DEVICE_LOOP
    with pytest.raises(ValueError):
        rd._opts(potential_mode="stored")
    with pytest.raises(ValueError):
        rd._opts(mode="fp16")


def test_bench_uses_the_traffic_summary_only_where_it_was_taken():
    """bench.py reports the committed ncu DRAM traffic only for the kernel source, workload and
    launch width it was captured on."""
    import json
    import sys

    sys.path.insert(0, ROOT)
    import bench

    d = json.load(open(os.path.join(ROOT, "profiles", "spmm_traffic.json")))
    w = d["width"]
    same_source = d["kernel_source_sha1"] == bench.kernel_source_hash()
    got = bench.load_traffic(d["workload"], w)
    assert got == (d["dram_bytes_per_launch"] if same_source else None)
    assert bench.load_traffic(d["workload"], w // 2) is None
    assert bench.load_traffic("chunglu1000000_128pairs", w) is None
