#!/usr/bin/env python3
"""Benchmark: resistance distance by batched Lanczos iteration on one GB300.

Workload: Chung-Lu power-law graph (n = 1,000,000 before the largest-component cut,
exponent 2.1, mean degree 20, 1e7 endpoint draws, unweighted) with 256 uniform random
(s,t) pairs answered in one batched query; FP32 vectors, FP64 alpha/beta/T_k; each pair
stops when its estimated relative error is below 1e-6; the true relative error of every
pair is then checked against the FP64 oracle (max_rel_err).

One step = one full query of the 256 pairs (every Lanczos step of every pair).
value = pairs/s over all ranks with the pair ids already on the device; e2e = the same
through the C ABI with host buffers (pinned pair ids in, host results out).

``--impl reference`` times the CPU oracle (plain C, FP64, one pair per thread) on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RD (s,t) pairs/sec at rel.err<=1e-6 (batched Lanczos, Chung-Lu 1M, 256 pairs)"
UNIT = "pairs/s"
REL_TOL = 1e-6
K_MAX = 200


KERNEL_NAMES = {1: "k_spmm (+ k_spmm_heavy)", 2: "k_spmm_rows (+ k_spmm_heavy)", 3: "k_spmm, degree order",
                4: "k_spmv_tasks", 5: "k_spmm_async (+ k_spmm_async_heavy)"}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha1()
    for f in ["spmm.cuh", "spmm_f32.cu"]:
        h.update(open(os.path.join(ROOT, "paper_2601_11159_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


def load_traffic(workload: str, width: int):
    """DRAM bytes of one SpMM launch pair (heavy-row pre-pass + main kernel) at the full width
    of the profiled pass, from the committed ncu summary, if it was taken on the current kernel
    source, on this workload and at this width, else None."""
    p = os.path.join(ROOT, "profiles", "spmm_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("kernel_source_sha1") != kernel_source_hash() or d.get("workload") != workload:
        return None
    if d.get("width") != width:
        return None
    return d.get("dram_bytes_per_launch")


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        # drain the pipe while the timed region runs (a full pipe would stall the sampler)
        self.reader = threading.Thread(target=lambda: self.lines.extend(self.proc.stdout), daemon=True)
        self.reader.start()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.reader.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in list(self.lines):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(backend: str = None):
    """One process per GPU (torchrun env). Ranks share nothing on the data path: each answers
    its own pairs; the process group only carries the barrier and the max of the timings."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def allmax(world, x: float) -> float:
    """Max over ranks of a host scalar (the slowest rank sets the job's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seed(rank: int) -> int:
    """Seed of rank r's pair set (weak scaling: every rank answers its own 256 pairs)."""
    from graphgen import workloads as W

    return W.BASE_SEED + 2 + 1000 * rank


def job_throughput(pairs_per_rank: int, world: int, steps: int, ms_max: float) -> float:
    """Whole-job pairs/s: all ranks' pairs over the slowest rank's time."""
    return pairs_per_rank * world * steps / (ms_max / 1000.0)


def workload(rank: int, n: int = 1_000_000, pairs: int = 256):
    from graphgen import workloads as W

    # the graph is the same on every rank (the seed of rank 0); the pairs are the rank's own
    g, _, _ = W.chunglu(n, 2.1, 20.0, n * 10, pairs, rank_seed(0))
    from graphgen import families as F

    s, t = F.random_pairs(g.n, pairs, rank_seed(rank))
    return g, s, t


CPU_STOP = 1e-9    # relative increment at which the timed CPU baseline stops (stricter than 1e-6)
REF_STOP = 1e-13   # relative increment of the oracle run that gives the reference values


def cpu_oracle(g, s, t, sample: int, threads: int = 0):
    """Timed CPU baseline: the oracle's -O3 build on `sample` pairs, one pair per thread."""
    from oracle import lanczos as O

    lib = O.load_timing()
    t0 = time.perf_counter()
    r, k, used = O.lanczos_batch(g, s[:sample], t[:sample], k_max=K_MAX, stop_tol=CPU_STOP, threads=threads,
                                 lib=lib)
    dt = time.perf_counter() - t0
    return r, k, used, dt


def oracle_reference(g, s, t):
    """Reference values for max_rel_err: the (pinned) oracle run to a relative increment of
    1e-13 on every pair (untimed)."""
    from oracle import lanczos as O

    r, _, _ = O.lanczos_batch(g, s, t, k_max=K_MAX, stop_tol=REF_STOP, threads=0)
    return r


def host_info() -> dict:
    """The host the oracle timings ran on: architecture, CPU model (x86 "model name", or the
    Arm implementer/part codes), logical CPUs."""
    import platform

    model = None
    try:
        fields = {}
        for line in open("/proc/cpuinfo"):
            if ":" in line:
                k, v = line.split(":", 1)
                fields.setdefault(k.strip(), v.strip())
        model = fields.get("model name") or (
            f"implementer {fields.get('CPU implementer')} part {fields.get('CPU part')}"
            if "CPU part" in fields else None)
    except OSError:
        pass
    return {"machine": platform.machine(), "model": model or platform.processor() or None,
            "nproc": os.cpu_count()}


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    g, s, t = workload(0)
    sample = args.ref_sample
    times = []
    for _ in range(args.warmup):
        cpu_oracle(g, s, t, min(sample, 4))
    used = 1
    for _ in range(args.steps):
        _, k, used, dt = cpu_oracle(g, s, t, sample)
        times.append(dt)
    total = sum(times)
    value = sample * len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * total / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "chunglu1m_256pairs", "n": g.n, "nnz": g.nnz, "pairs_per_step": sample,
                   "sample": f"{sample} of the 256 pairs per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "host": host_info(),
                         "build": "gcc -O3 -fopenmp",
                         "sample": f"{sample} pairs of the 256-pair workload per step, stop at relative "
                                   f"increment {CPU_STOP:g}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def profile_config(rd, name, call="query"):
    """One SpMM-heavy query of a workload inside cudaProfilerStart/Stop, after a warm-up query
    (which also runs the autotuner), for ncu --profile-from-start off: 4 fixed Lanczos steps
    over all of the workload's pairs (double-float vectors for the road grid; for grid64 the
    bench line's single-pair query: FP64, residual 1e-10, one whole-recurrence launch). With
    call="grad": instead the configs sweep's gradient call (rd_edge_grad over all of the
    workload's pairs, rel_tol 1e-6, k_max 200, upstream gradient 1), after a warm-up call."""
    import torch

    from graphgen import workloads as W

    make = {"chunglu1m": W.chunglu1m, "rmat24": W.rmat24, "roadgrid4096": W.roadgrid4096,
            "chunglu4m_w": W.chunglu4m_w, "grid64": W.grid64,
            # a small road grid (1024^2, 64 pairs at distance 256) for multi-pass ncu captures
            "roadgrid1024": lambda: W.roadgrid(1024, 64, 256)}[name]
    g, s, t = make()
    G = rd.Graph.from_csr(g)
    sd, td = torch.from_numpy(s).cuda(), torch.from_numpy(t).cuda()
    mode = "df64" if name.startswith("roadgrid") else "fp32"
    if name == "grid64":  # the single-pair latency workload as the bench line runs it
        mode = "fp64"
        kw = dict(mode=mode, k_max=500, rel_tol=0.0, resid_tol=1e-10)
        run = lambda: G.query(s, t, **kw)  # noqa: E731
    elif call == "grad":
        ones = torch.ones(len(s), dtype=torch.float64, device="cuda")
        mode = "fp32"
        kw = dict(mode=mode, k_max=200, rel_tol=1e-6, device_loop=False)
        run = lambda: G.edge_grad(sd, td, ones, **kw)  # noqa: E731
    else:
        # host-driven steps: ncu lists no kernels launched from a conditional graph node's body
        kw = dict(mode=mode, k_max=4, fixed_k=True, device_loop=False)
        run = lambda: G.query(sd, td, **kw)  # noqa: E731
    run()
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    run()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    st = G.last_stats()
    print(json.dumps({"profiled": name, "call": call, "mode": mode, "n": g.n, "nnz": g.nnz, "pairs": len(s),
                      "rhs_tile": st["rhs_tile"], "kernel": st["kernel"], "spmm_bytes_per_launch":
                      st["spmm_bytes"] / max(st["spmm_launches"], 1)}), flush=True)
    G.close()


def run_config_sweep(rd, timed, only=None):
    """One JSON line per synthetic workload (sizes and recipes in graphgen/workloads.py), or only
    the one named by `only`:
    grid64       -- one pair (corner to corner), FP64, plain single-vector path, stop at relative
                    residual 1e-10; error against the dense pseudo-inverse;
    chunglu1m    -- 256 pairs, FP32 vectors, rel_tol 1e-6: batched vs plain (16 pairs) pairs/s;
                    error against the FP64 oracle on 32 sampled pairs;
    roadgrid4096 -- 64 pairs, double-float vectors (FP64-class), rel_tol 1e-6 (the FP32-vector floor
                    at this condition number is about 5e-5, so FP32 runs to relative residual 1e-6
                    for time only); error of 4 pairs against the same pairs run to relative
                    residual 1e-10;
    chunglu4m_w  -- 32 pairs, gradient over all edges (rd_edge_grad, FP32 vectors, device in and
                    out), gradients/s and the forward error against the oracle on 4 pairs;
    rmat24       -- 128 pairs, FP32 vectors, rel_tol 1e-6: batched vs plain (8 pairs) pairs/s;
                    error against the oracle on 8 sampled pairs."""
    import torch

    from graphgen import workloads as W
    from oracle import dense
    from oracle import lanczos as O

    def want(name):
        return only is None or only == name

    def line(**kw):
        print(json.dumps(dict(sweep="configs", **kw)), flush=True)

    def rel(a, b):
        return float(np.max(np.abs(np.asarray(a, np.float64) / np.asarray(b, np.float64) - 1)))

    if want("grid64"):
        g, s, t = W.grid64()
        G = rd.Graph.from_csr(g)
        exact = dense.DenseRD.of(g).r(s, t)
        ms, res = timed(lambda: G.query(s, t, mode="fp64", k_max=500, rel_tol=0.0, resid_tol=1e-10, plain=True))
        line(workload="grid64", pairs=1, mode="fp64", path="plain", query_ms=ms, pairs_per_s=1e3 / ms,
             iters=int(res.iters[0]), max_rel_err=rel(res.r, exact))
        G.close()

    for name, make, pairs_plain in [("chunglu1m", W.chunglu1m, 16), ("rmat24", W.rmat24, 8)]:
        if not want(name):
            continue
        g, s, t = make()
        G = rd.Graph.from_csr(g)
        sd, td = torch.from_numpy(s).cuda(), torch.from_numpy(t).cuda()
        kw = dict(mode="fp32", k_max=200, rel_tol=1e-6)
        ms_b, rb = timed(lambda: G.query(sd, td, **kw))
        ms_p, rp = timed(lambda: G.query(sd[:pairs_plain], td[:pairs_plain], plain=True, **kw), reps=2)
        idx = np.linspace(0, len(s) - 1, 32 if name == "chunglu1m" else 8).astype(int)
        ref, _, _ = O.lanczos_batch(g, s[idx], t[idx], k_max=200, stop_tol=1e-13, threads=0)
        rbn, rpn = rb.r.cpu().numpy(), rp.r.cpu().numpy()
        pidx = idx[idx < pairs_plain]
        line(workload=name, n=g.n, nnz=g.nnz, pairs=len(s), mode="fp32",
             batched_pairs_per_s=len(s) / (ms_b / 1e3), plain_pairs_per_s=pairs_plain / (ms_p / 1e3),
             batched_over_plain=(len(s) / ms_b) / (pairs_plain / ms_p),
             iters_median=float(np.median(rb.iters.cpu().numpy())), iters_max=int(rb.iters.max()),
             max_rel_err_batched=rel(rbn[idx], ref),
             max_rel_err_plain=rel(rpn[pidx], ref[np.isin(idx, pidx)]) if len(pidx) else None,
             sampled_pairs=len(idx))
        G.close()

    if want("roadgrid4096"):
        g, s, t = W.roadgrid4096()
        G = rd.Graph.from_csr(g)
        msdf, rdf = timed(lambda: G.query(s, t, mode="df64", k_max=40000, rel_tol=1e-6), reps=1)
        ms32, r32 = timed(lambda: G.query(s, t, mode="fp32", k_max=40000, rel_tol=0.0, resid_tol=1e-6), reps=1)
        tight = G.query(s[:4], t[:4], mode="df64", k_max=60000, rel_tol=0.0, resid_tol=1e-10)
        line(workload="roadgrid4096", n=g.n, nnz=g.nnz, pairs=len(s),
             df64_rel_tol_1e6={"query_ms": msdf, "pairs_per_s": len(s) / (msdf / 1e3),
                               "iters_median": float(np.median(rdf.iters)), "iters_max": int(rdf.iters.max()),
                               "max_rel_err_vs_resid1e-10": rel(rdf.r[:4], tight.r)},
             fp32_resid_1e6={"query_ms": ms32, "pairs_per_s": len(s) / (ms32 / 1e3),
                             "iters_median": float(np.median(r32.iters)), "iters_max": int(r32.iters.max()),
                             "max_rel_err_vs_resid1e-10": rel(r32.r[:4], tight.r)},
             reference_iters=tight.iters.tolist())
        G.close()

    if want("chunglu4m_w"):
        g, s, t = W.chunglu4m_w()
        G = rd.Graph.from_csr(g)
        sd, td = torch.from_numpy(s).cuda(), torch.from_numpy(t).cuda()
        ones = torch.ones(len(s), dtype=torch.float64, device="cuda")
        # device in, device out: the gradient (one float per stored entry) stays in HBM
        ms_g, (gw, r) = timed(lambda: G.edge_grad(sd, td, ones, mode="fp32", k_max=200, rel_tol=1e-6), reps=2)
        ms_f, rf = timed(lambda: G.query(sd, td, mode="fp32", k_max=200, rel_tol=1e-6), reps=2)
        idx = np.array([0, 9, 21, 30])
        ref, _, _ = O.lanczos_batch(g, s[idx], t[idx], k_max=200, stop_tol=1e-13, threads=0)
        line(workload="chunglu4m_w", n=g.n, nnz=g.nnz, pairs=len(s), mode="fp32",
             gradient_ms=ms_g, gradients_per_s=len(s) / (ms_g / 1e3), forward_ms=ms_f,
             gradient_over_forward=ms_g / ms_f, max_rel_err_r=rel(r.cpu().numpy()[idx], ref),
             grad_entries=int(gw.numel()))
        G.close()


def condition_number(g, tol: float = 1e-6):
    """kappa = 2/(1 - mu_2), mu_2 the second-largest eigenvalue of Ahat = D^{-1/2} W D^{-1/2}
    (the largest is 1, eigenvector D^{1/2} 1, deflated here): scipy eigsh on the host, FP64."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla

    w = np.ones(g.nnz) if g.w is None else g.w.astype(np.float64)
    A = sp.csr_matrix((w, g.col, g.row_ptr), shape=(g.n, g.n))
    d = np.asarray(A.sum(axis=1)).ravel()
    isd = 1.0 / np.sqrt(d)
    Ah = sp.diags(isd) @ A @ sp.diags(isd)
    u = np.sqrt(d) / np.linalg.norm(np.sqrt(d))
    op = sla.LinearOperator(Ah.shape, matvec=lambda x: Ah @ x - u * (u @ x), dtype=np.float64)
    mu2 = float(sla.eigsh(op, k=1, which="LA", tol=tol, return_eigenvectors=False, maxiter=20000).max())
    return mu2, 2.0 / (1.0 - mu2)


def run_kappa(only=None):
    """Condition numbers of the synthetic workloads (host only). The road grid's gap (about
    1e-7) is beyond eigsh in reasonable time: its line gives the undeleted 4096^2 grid's value
    8 N^2 / pi^2 (mu_2 = 1 - pi^2/(4 N^2) to leading order) as an estimate."""
    import math

    from graphgen import workloads as W

    for name, make in (("grid64", W.grid64), ("chunglu1m", W.chunglu1m), ("chunglu4m_w", W.chunglu4m_w),
                       ("rmat24", W.rmat24)):
        if only and name != only:
            continue
        g = make()[0]
        t0 = time.time()
        mu2, kappa = condition_number(g)
        print(json.dumps({"sweep": "kappa", "workload": name, "n": g.n, "nnz": g.nnz, "mu2": mu2, "kappa": kappa,
                          "method": "eigsh (deflated Ahat)", "host_s": round(time.time() - t0, 1)}), flush=True)
    if not only or only == "roadgrid4096":
        N = 4096
        print(json.dumps({"sweep": "kappa", "workload": "roadgrid4096", "kappa": 8 * N * N / math.pi ** 2,
                          "method": "estimate: undeleted 4096^2 grid, 8 N^2 / pi^2"}), flush=True)


def run_sweeps(which: str, only=None, profile=False, profile_call="query"):
    """Extra measurements beyond the main line (one JSON line each):
    scaling  -- Erdos-Renyi and Barabasi-Albert graphs, n = 1e2..1e6, m = n ln n, k = 20 fixed,
                64 pairs, FP32 (the scalability experiment, Exp-3);
    density  -- Erdos-Renyi n = 1000 with average degree 5/25/50/250, 10 top-degree vs 10
                random vertices (all ordered pairs), k = 15 / k = 5, absolute error against the
                dense oracle (the s,t-selection and density experiment, Exp-6);
    pm       -- steps and time to relative error 1e-6 for the Lanczos iteration and the Power
                Method (Algorithm 1) on a road-like grid and on a Chung-Lu graph;
    configs  -- the five synthetic workloads: pairs/s of the batched and the plain path at
                relative error 1e-6 (gradients/s for the weighted Chung-Lu case), each with its
                measured error (see run_config_sweep)."""
    import torch

    import paper_2601_11159_gb300 as rd
    from graphgen import families as F
    from oracle import dense
    from oracle import lanczos as O

    def timed(fn, reps=3):
        best, out = None, None
        for _ in range(reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = fn()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        return best, out

    if which in ("scaling", "all"):
        import math

        for fam in ["er", "ba"]:
            for n in [100, 1000, 10_000, 100_000, 1_000_000]:
                m = int(n * math.log(n))
                g = F.erdos_renyi(n, m, 7) if fam == "er" else F.barabasi_albert(n, max(1, int(round(math.log(n)))), 7)
                s, t = F.random_pairs(g.n, 64, 8)
                G = rd.Graph.from_csr(g)
                sd, td = torch.from_numpy(s).cuda(), torch.from_numpy(t).cuda()
                ms, res = timed(lambda: G.query(sd, td, mode="fp32", k_max=20, fixed_k=True))
                ref, _, _ = O.lanczos_batch(g, s[:4], t[:4], k_max=400, stop_tol=1e-13, threads=0)
                err = np.abs(res.r.cpu().numpy()[:4] - ref) / ref
                print(json.dumps({"sweep": "scaling", "family": fam, "n": g.n, "m": g.nnz // 2, "k": 20, "pairs": 64,
                                  "query_ms": ms, "pairs_per_s": 64 / (ms / 1000), "max_rel_err_k20": float(err.max())}),
                      flush=True)
                G.close()
    if which in ("density", "all"):
        for d in [5, 25, 50, 250]:
            g = F.erdos_renyi(1000, 1000 * d // 2, 11)
            deg = np.diff(g.row_ptr)
            top = np.argsort(-deg, kind="stable")[:10]
            rnd = F.random_pairs(g.n, 10, 12)[0]
            D = dense.DenseRD.of(g)
            G = rd.Graph.from_csr(g)
            for label, vs in [("top_degree", top), ("random", rnd)]:
                a, b = np.meshgrid(vs, vs)
                keep = a != b
                s, t = a[keep].astype(np.int32), b[keep].astype(np.int32)
                exact = D.r(s, t)
                for k in [5, 15]:
                    r = G.query(s, t, mode="fp64", k_max=k, fixed_k=True).r
                    print(json.dumps({"sweep": "density", "n": g.n, "avg_degree": d, "select": label, "k": k,
                                      "mean_abs_err": float(np.mean(np.abs(r - exact))),
                                      "max_abs_err": float(np.max(np.abs(r - exact)))}), flush=True)
            G.close()
    if which in ("configs", "all"):
        if profile:
            profile_config(rd, only or "chunglu1m", profile_call)
        else:
            run_config_sweep(rd, timed, only)
    if which in ("pm", "all"):
        from graphgen import workloads as W

        cases = []
        gg = F.grid_deleted(128, 0.05, 3)
        cases.append(("grid128_del5", gg) + F.random_pairs(gg.n, 8, 5))
        cases.append(("chunglu100k",) + W.chunglu(100_000, 2.1, 20.0, 1_000_000, 8, 9))
        for name, g, s, t in cases:
            G = rd.Graph.from_csr(g)
            ref, _, _ = O.lanczos_batch(g, s, t, k_max=20000, stop_tol=1e-14, threads=0)
            steps = 200_000 if name.startswith("grid") else 2000
            _, hist = G.power_method(s, t, steps, mode="fp64", history=True)
            rel_pm = np.abs(hist / ref[None, :] - 1)
            k_pm = [int(np.argmax(rel_pm[:, p] <= 1e-6)) if np.any(rel_pm[:, p] <= 1e-6) else None
                    for p in range(len(s))]
            kmax_pm = max(k for k in k_pm if k is not None) if any(k is not None for k in k_pm) else steps
            ms_pm, _ = timed(lambda: G.power_method(s, t, kmax_pm, mode="fp64"), reps=1)
            ms_lz, res = timed(lambda: G.query(s, t, mode="fp64", k_max=20000, rel_tol=1e-7))
            err_lz = float(np.max(np.abs(res.r / ref - 1)))
            print(json.dumps({"sweep": "lanczos_vs_power_method", "graph": name, "n": g.n, "pairs": len(s),
                              "lanczos_steps_max": int(res.iters.max()), "lanczos_ms": ms_lz,
                              "lanczos_max_rel_err": err_lz, "pm_steps_to_1e-6": k_pm, "pm_ms": ms_pm,
                              "pm_steps_run": kmax_pm}), flush=True)
            G.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-sample", type=int, default=32)
    ap.add_argument("--cpu-sample", type=int, default=256)
    ap.add_argument("--plain-sample", type=int, default=16)
    ap.add_argument("--cpu1-sample", type=int, default=8, help="pairs of the one-core oracle timing")
    ap.add_argument("--prof-steps", type=int, default=5,
                    help="queries of the separate profiled pass that times the SpMM launches")
    ap.add_argument("--profile-pass-range", action="store_true",
                    help="bracket the first query of the profiled pass with cudaProfilerStart/Stop")
    ap.add_argument("--no-device-loop", action="store_true",
                    help="run the steps from the host-driven loop (for a per-kernel ncu launch list: ncu "
                         "does not list kernels launched from a conditional graph node's body)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--n", type=int, default=1_000_000, help="graph size (smaller only for profiling)")
    ap.add_argument("--pairs", type=int, default=256)
    ap.add_argument("--kernel", default="tuned", choices=["tuned", "group", "stream"])
    ap.add_argument("--rhs-tile", type=int, default=0)
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the timed region with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    ap.add_argument("--only", default=None,
                    choices=["grid64", "chunglu1m", "rmat24", "roadgrid4096", "chunglu4m_w", "roadgrid1024"],
                    help="with --sweep configs: one workload; with --profile-range: a short profiled query of it "
                         "(roadgrid1024: profiling only)")
    ap.add_argument("--profile-call", default="query", choices=["query", "grad"],
                    help="with --sweep configs --profile-range: the profiled call (grad: rd_edge_grad)")
    ap.add_argument("--sweep", default=None, choices=["scaling", "density", "pm", "configs", "kappa", "all"],
                    help="extra measurements instead of the main line (kappa: host only)")
    args = ap.parse_args()
    if args.sweep == "kappa":
        return run_kappa(args.only)
    if args.sweep:
        return run_sweeps(args.sweep, args.only, args.profile_range, args.profile_call)
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch

    torch.cuda.set_device(local)
    import paper_2601_11159_gb300 as rd
    from paper_2601_11159_gb300 import build as B

    if not os.path.exists(B.LIB):
        B.build()
    g, s_np, t_np = workload(rank, args.n, args.pairs)
    P = s_np.size
    G = rd.Graph.from_csr(g)
    s_dev = torch.from_numpy(s_np).cuda()
    t_dev = torch.from_numpy(t_np).cuda()
    opts = dict(mode="fp32", k_max=K_MAX, rel_tol=REL_TOL, kernel=args.kernel, rhs_tile=args.rhs_tile)
    if args.no_device_loop:  # the same kernels launched step by step (ncu lists them one by one)
        opts["device_loop"] = False
    stream = torch.cuda.current_stream()

    # warm-up (also settles the workspace)
    for _ in range(args.warmup):
        res = G.query(s_dev, t_dev, **opts)
    torch.cuda.synchronize()

    # device-resident timed region
    clk = Clocks(local)
    clk.start()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    spmm_ms = 0.0
    spmm_n = 0
    spmm_bytes = 0.0
    steps_max = 0
    compactions = 0
    if args.profile_range:
        torch.cuda.profiler.start()
    # the shipped configuration: CUDA-graph replay of the steps, no event timing inside
    e0.record(stream)
    for _ in range(args.steps):
        res = G.query(s_dev, t_dev, **opts)
        st = G.last_stats()
        launches += st["launches"]
        steps_max = max(steps_max, st["steps"])
        compactions += st["compactions"]
    e1.record(stream)
    torch.cuda.synchronize()
    if args.profile_range:
        torch.cuda.profiler.stop()
    barrier(world)
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    ms_max = allmax(world, ms)
    value = job_throughput(P, world, args.steps, ms_max)
    # a separate profiled pass gives the dominant kernel's launch times: the same query with
    # CUDA events around every SpMM launch pair on the library's stream (launch-per-kernel
    # loop) and without column compaction, so that every SpMM launch is the full-width one
    # whose algorithmic bytes and DRAM traffic the roofline compares
    for i in range(args.prof_steps):
        if args.profile_pass_range and i == 0:
            torch.cuda.profiler.start()
        G.query(s_dev, t_dev, profile=True, compact=False, **opts)
        if args.profile_pass_range and i == 0:
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
        sp = G.last_stats()
        spmm_ms += sp["spmm_ms"]
        spmm_n += sp["spmm_launches"]
        spmm_bytes += sp["spmm_bytes"]
    torch.cuda.synchronize()
    r_gpu = res.r.cpu().numpy()
    iters = res.iters.cpu().numpy()
    status = res.status.cpu().numpy()

    # end to end: host (pinned) pair ids in, host results out, copies inside the timed region
    e2e_value = None
    plain_value = None
    plain_r = None
    if not args.no_e2e:
        e2e_value = run_e2e(G, s_np, t_np, opts, args, world)
    if not args.no_plain:
        plain_value, plain_r = run_plain(G, s_dev, t_dev, opts, args, stream)
    st["compactions_per_query"] = compactions / args.steps
    st["grid64"] = run_grid64() if rank == 0 and not args.no_plain else None
    return finish(args, world, rank, g, P, value, ms_max, res, r_gpu, iters, status, st, launches, spmm_ms,
                  spmm_n, spmm_bytes, steps_max, clocks, e2e_value, plain_value, plain_r, s_np, t_np)


def run_grid64(reps: int = 20) -> dict:
    """The single-pair latency workload: 64x64 grid, corner to opposite corner, FP64, relative
    residual 1e-10 (k <= 500), on the shipped path (the whole-recurrence kernel, here on a
    thread-block cluster); error against the exact spectral sum."""
    import torch

    import paper_2601_11159_gb300 as rd
    from graphgen import workloads as W
    from tests import closed_forms as CF

    g, s, t = W.grid64()
    ref = CF.grid_r(64, 64, 0, 4095)
    G = rd.Graph.from_csr(g)
    kw = dict(mode="fp64", k_max=500, rel_tol=0.0, resid_tol=1e-10)
    for _ in range(3):
        r = G.query(s, t, **kw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        r = G.query(s, t, **kw)
    torch.cuda.synchronize()
    ms = 1e3 * (time.perf_counter() - t0) / reps
    st = G.last_stats()
    k = int(r.iters[0])
    return {"workload": "grid64 corner pair (n = 4096), FP64, residual 1e-10", "ms_per_query": ms,
            "steps": k, "us_per_step": 1e3 * ms / k, "rel_err_vs_closed_form": abs(float(r.r[0]) - ref) / ref,
            "ctas_per_pair": int(st["onchip_ctas"]), "timing": f"host clock over {reps} queries (host ids in, "
            "host result out)"}


def run_e2e(G, s_np, t_np, opts, args, world):
    import torch

    P = s_np.size
    s_h = torch.from_numpy(s_np).pin_memory()
    t_h = torch.from_numpy(t_np).pin_memory()
    for _ in range(2):
        G.query(s_h, t_h, **opts)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        re2e = G.query(s_h, t_h, **opts)
    torch.cuda.synchronize()
    e2e_s = allmax(world, time.perf_counter() - t0)
    assert isinstance(re2e.r, np.ndarray)
    return P * world * args.steps / e2e_s


def run_plain(G, s_dev, t_dev, opts, args, stream):
    """The plain one-pair-per-launch path on a sample of the same pairs."""
    import torch

    P = s_dev.numel()
    ps = min(args.plain_sample, P)
    for _ in range(2):
        G.query(s_dev[:2], t_dev[:2], plain=True, **opts)
    torch.cuda.synchronize()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    rp = G.query(s_dev[:ps], t_dev[:ps], plain=True, **opts)
    p1.record(stream)
    torch.cuda.synchronize()
    return ps / (p0.elapsed_time(p1) / 1000.0), rp.r.cpu().numpy()


def finish(args, world, rank, g, P, value, ms_max, res, r_gpu, iters, status, st, launches, spmm_ms, spmm_n,
           spmm_bytes, steps_max, clocks, e2e_value, plain_value, plain_r, s_np, t_np):
    if rank != 0:
        return 0

    peak, peak_kind = load_peaks()
    # SpMM launches shrink as converged pairs are packed: total algorithmic bytes over total time
    avg_launch_ms = spmm_ms / max(spmm_n, 1)
    achieved = spmm_bytes / (spmm_ms / 1000.0) / 1e9 if spmm_n and spmm_ms > 0 else None
    workload_name = "chunglu1m_256pairs" if args.n == 1_000_000 and P == 256 else f"chunglu{args.n}_{P}pairs"
    traffic = load_traffic(workload_name, P)

    cpu = None
    max_rel = None
    if not args.no_cpu:
        cs = min(args.cpu_sample, P)
        r_or, k_or, used, dt = cpu_oracle(g, s_np, t_np, cs)
        r_ref = oracle_reference(g, s_np, t_np)
        rel = np.abs(r_gpu - r_ref) / np.abs(r_ref)
        max_rel = float(rel.max())
        cpu = {"value": cs / dt, "unit": UNIT, "cores": int(used), "kind": "oracle", "host": host_info(),
               "build": "gcc -O3 -fopenmp (no -march=native: host code builds alike on x86 and Arm)",
               "sample": f"{cs} of the {P} pairs, FP64 C Lanczos, stop at relative increment {CPU_STOP:g}",
               "reference": f"max_rel_err over all {P} pairs against the oracle run to a relative increment "
                            f"of {REF_STOP:g}",
               "max_rel_err_gpu_vs_oracle": max_rel, "median_rel_err_gpu_vs_oracle": float(np.median(rel))}
        if plain_r is not None:
            ps = plain_r.size
            cpu["max_rel_err_plain_vs_oracle"] = float((np.abs(plain_r - r_ref[:ps]) / np.abs(r_ref[:ps])).max())
        # one core (the paper's setting: one CPU thread), on a smaller sample of the same pairs
        _, _, _, dt1 = cpu_oracle(g, s_np, t_np, args.cpu1_sample, threads=1)
        cpu["single_core"] = {"value": args.cpu1_sample / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"{args.cpu1_sample} of the {P} pairs"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name, "n": g.n, "nnz": g.nnz, "pairs": P, "kernel": int(st["kernel"]),
                   "precision": "FP32 vectors and SpMM, FP64 alpha/beta/T_k and reductions",
                   "stop": f"estimated relative error <= {REL_TOL}", "k_max": K_MAX,
                   "lanczos_steps_max": int(steps_max), "iters_median": float(np.median(iters)),
                   "rhs_tile": int(st["rhs_tile"]), "rows_per_warp": int(st["rows_per_warp"]),
                   "compactions_per_query": st["compactions_per_query"],
                   "l2": "inputs larger than L2 (two 1 GB vector blocks per query)",
                   "parallelism": f"replicas x{world}, pairs sharded, no collective",
                   "all_pairs_ok": bool(np.all(status >= 0))},
        "e2e": None if e2e_value is None else {"value": e2e_value, "unit": UNIT,
                                               "h2d_bytes_per_step": int(2 * 4 * P),
                                               "d2h_bytes_per_step": int(24 * P)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "kernel": KERNEL_NAMES.get(int(st["kernel"]), "spmm"),
                     "peak_kind": f"{peak_kind} hbm_gbs (copy)",
                     "timing": f"CUDA events around each SpMM launch pair on the library's stream, in a "
                               f"separate profiled pass of {args.prof_steps} queries without column "
                               f"compaction (every SpMM launch at the full {P}-column width); value and "
                               f"e2e are timed on the CUDA-graph path without events",
                     "algorithmic_bytes_per_launch": spmm_bytes / max(spmm_n, 1), "avg_launch_ms": avg_launch_ms,
                     "launches_timed": spmm_n,
                     # DRAM bytes actually moved per launch (ncu, profiles/) over the live launch time
                     "dram_gbs": traffic / (avg_launch_ms / 1e3) / 1e9 if traffic and avg_launch_ms else None,
                     "dram_frac": traffic / (avg_launch_ms / 1e3) / 1e9 / peak if traffic and avg_launch_ms else None},
        "plain_pairs_per_s": plain_value,
        "batched_over_plain": None if plain_value is None else value / world / plain_value,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "max_rel_err": max_rel,
        "single_pair_latency": st.get("grid64"),
    }
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
