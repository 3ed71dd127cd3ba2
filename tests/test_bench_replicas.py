"""The benchmark's multi-rank logic on CPU (gloo, world size 2).

The hashing path has no exchange step, so several GPUs run independent
replicas: each rank hashes its own seeded data, the slowest rank's time sets
the job time, and the whole-job throughput counts every rank's bytes.  These
tests run that logic with two gloo processes on the CPU, and run the
reference arm (the CPU oracle) under torchrun with two ranks, where rank 0
alone prints the result line.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, ws, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        seconds = [1.5, 2.5][rank]                     # rank 1 is the slower replica
        t = bench.max_over_ranks(seconds, dist, "cpu")
        host = bench.sliding_workload(bench.rank_seed(7, rank), 2, 4096)
        q.put((rank, t, bench.aggregate_gbs(ws, 256 << 20, 10, t), host[:64].tobytes()))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_max_time_and_aggregate():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, v0, h0), (r1, t1, v1, h1) = res
    assert t0 == t1 == 2.5                             # both ranks see the slowest time
    assert v0 == v1 == pytest.approx(2 * (256 << 20) * 10 / 2.5 / 1e9)
    assert h0 != h1                                    # each replica has its own data


def test_reference_arm_under_torchrun_rank0_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--units", "2",
           "--unit-bytes", "65536", "--cpu-units", "2"]
    p = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GB/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["n_gpus"] == 2
