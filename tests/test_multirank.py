"""The multi-rank path of bench.py on CPU ranks (gloo, world size 2).

Every GB300 machine here has one GPU, so N > 1 runs independent replicas, one per
rank (the sweep needs no exchange between replicas).  These tests check the
host-side parts of that path: the max-over-ranks time, the sum of attempts
over ranks, and that under torchrun only rank 0 prints the reference line.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

import torch.distributed as dist
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=2)
    t = bench.max_over_ranks(dist, 1.5 + rank)
    n = bench.sum_over_ranks(dist, 1000.0 * (rank + 1))
    out.put((rank, t, n))
    dist.barrier()
    dist.destroy_process_group()


def test_max_and_sum_over_two_gloo_ranks():
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, n in res:
        assert t == 2.5       # the slowest rank's time
        assert n == 3000.0    # attempts of all ranks


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "3", "--workload", "cpm2d_200"]
    env = dict(os.environ, CPM_BENCH_BACKEND="gloo", OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
