"""The multi-GPU form of the benchmark on CPU: two gloo ranks, each with its own pair set
(pairs shard across ranks, the graph is replicated, no collective on the data path); the
job's time is the max over ranks."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    w, r, _ = bench.dist_setup("gloo")
    assert (w, r) == (world, rank)
    from graphgen import families as F

    g = F.grid(20)
    s, t = F.random_pairs(g.n, 16, bench.rank_seed(r))
    my_ms = 100.0 + 50.0 * r                      # rank 1 is the slower one
    ms_max = bench.allmax(w, my_ms)
    bench.barrier(w)
    out.put((r, s.tolist(), t.tolist(), ms_max, bench.job_throughput(16, w, 10, ms_max)))
    import torch.distributed as dist

    dist.destroy_process_group()


def test_two_gloo_ranks_shard_pairs_and_take_max_time():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, t0, m0, v0), (r1, s1, t1, m1, v1) = res
    assert m0 == m1 == 150.0                       # both ranks see the slowest rank's time
    assert v0 == v1 == pytest.approx(16 * 2 * 10 / 0.150)
    assert (s0, t0) != (s1, t1)                    # different pairs on each rank


def test_reference_arm_prints_one_json_line():
    """bench.py --impl reference times the CPU oracle on a bounded sample of the bench
    workload and prints one JSON line with the contract's keys (runs on CPU, no GPU)."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PYTHONPATH=root)
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3", "--ref-sample", "2"], capture_output=True, text=True, env=env,
                         timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
