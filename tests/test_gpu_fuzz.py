"""Seeded random jobs over every parameter the path takes, against the CPU
oracle, bit-exact: the four kinds (MD5 and SHA-1, direct and sliding), unit
sizes from 0 bytes to a few hundred KiB (log-uniform, plus the padding and
tile edges), segment sizes from 1 byte to 64 KiB, windows of 1 to 55 bytes,
masks of 0 to 10 bits with random targets (mask 0: a boundary at every
offset), chunk segment sizes from 16 bytes up, input misalignments 0-15 and
output buffers that are sometimes too small (CRYSTAL_EOVERFLOW: header and
bitmap still exact).  Once through the stateless launchers on one device
batch, once through the job runtime with graphs and random launch geometry
per size class."""
import concurrent.futures as cf
import os

import numpy as np
import pytest

from helpers import first_difference, same_result

pytestmark = pytest.mark.gpu

EDGE_SIZES = [0, 1, 19, 20, 21, 55, 56, 63, 64, 65, 119, 120, 2047, 2048, 2049, 4095, 4096, 4097, 2068]


@pytest.fixture(scope="module")
def C():
    import torch

    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    from paper_1005_1695_b300 import crystal

    crystal.load()
    return crystal


def _random_jobs(C, seed, count):
    """(kind, bytes, out_size, params, misalignment) per job, all seeded."""
    rng = np.random.default_rng(seed)
    jobs = []
    for i in range(count):
        kind = int(rng.integers(1, 5))
        n = int(EDGE_SIZES[i % len(EDGE_SIZES)]) if i % 3 == 0 else int(np.exp(rng.uniform(0, np.log(300_000))))
        data = rng.integers(0, 256, n, dtype=np.uint8)
        if kind in (2, 4) and n > 4096 and rng.random() < 0.5:
            # repeated 1 KiB blocks: equal content gives equal boundaries
            block = rng.integers(0, 256, 1024, dtype=np.uint8)
            for o in range(0, n - 1024, 2048):
                data[o:o + 1024] = block
        seg = int(rng.choice([1, 7, 64, 100, 333, 1024, 4096, 65536]))
        w = int(rng.integers(1, 56))
        bits = int(rng.integers(0, 11))
        mask = 0
        for b in rng.choice(32, size=bits, replace=False):
            mask |= 1 << int(b)
        target = int(rng.integers(0, 1 << 32)) & mask
        cseg = int(rng.choice([16, 64, 1000, 4096]))
        p = C.params(segment_bytes=seg, window_bytes=w, mask=mask, target=target, chunk_segment_bytes=cseg)
        if kind in (2, 4):
            worst = C.out_bytes(kind, n, p)
            # a quarter of the sliding jobs get room for only a few chunks
            out = C.sliding_out_bytes(n, int(rng.integers(0, 8)), kind) if rng.random() < 0.25 else worst
        else:
            out = C.digest_size(kind)
        jobs.append((kind, data, out, p, int(rng.integers(0, 16))))
    return jobs


def _oracle(oracle_mod, jobs):
    def one(j):
        kind, data, out, p, _ = j
        return oracle_mod.task(kind, data.tobytes(), out, seg_bytes=p.segment_bytes, window=p.window_bytes,
                               mask=p.mask, target=p.target, chunk_seg_bytes=p.chunk_segment_bytes)

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        return list(ex.map(one, jobs))


def _compare(jobs, got, want, what):
    for i, ((kind, data, _, p, _), g, (st, w)) in enumerate(zip(jobs, got, want)):
        assert st in (0, 1), (what, i, st)
        assert same_result(kind, len(data), g, w), \
            f"{what} job {i} (kind {kind}, n {len(data)}, S {p.segment_bytes}, w {p.window_bytes}, " \
            f"mask {p.mask:#x}): " + first_difference(kind, len(data), g, w)


@pytest.mark.parametrize("seed", [101, 202, 303])
def test_fuzz_device_batch(C, oracle_mod, seed):
    import torch

    jobs = _random_jobs(C, seed, 120)
    pos, offs = 0, []
    for kind, data, out, p, mis in jobs:
        pos = (pos + 255) // 256 * 256 + mis
        offs.append(pos)
        pos += len(data)
    host = np.zeros(pos + 256, dtype=np.uint8)
    for o, (_, data, _, _, _) in zip(offs, jobs):
        host[o:o + len(data)] = data
    d_in = torch.from_numpy(host).cuda()
    b = C.DeviceBatch(d_in, offs, [len(j[1]) for j in jobs], [j[0] for j in jobs], out_sizes=[j[2] for j in jobs],
                      per_unit_params=[j[3] for j in jobs])
    b.launch()
    torch.cuda.synchronize()
    assert b.device_status() == 0
    _compare(jobs, b.outputs(), _oracle(oracle_mod, jobs), "batch")


@pytest.mark.parametrize("seed", [404, 505])
def test_fuzz_job_runtime(C, oracle_mod, seed):
    jobs = _random_jobs(C, seed, 150)
    want = _oracle(oracle_mod, jobs)
    rng = np.random.default_rng(seed + 1)
    with C.Context(max_in_bytes=300_000, max_out_bytes=max(j[2] for j in jobs), device_pool_bytes=1 << 30,
                   host_pool_bytes=1 << 30, n_streams=int(rng.integers(1, 6)),
                   max_batch_jobs=int(rng.integers(1, 20)), flags=C.CRYSTAL_FLAG_GRAPHS) as ctx:
        for cls in range(C.CRYSTAL_SIZE_CLASSES):
            ctx.set_geometry(cls, C.geometry(seg_threads=int(rng.choice([64, 128, 256])),
                                             win_ctas_per_sm=int(rng.choice([0, 2, 4])),
                                             win_registers=int(rng.choice([32, 64]))))
        tasks = []
        for kind, data, out, p, _ in jobs:
            t = ctx.task_create(len(data), out)
            if len(data):
                t.h_in[:] = data
            assert t.submit(kind, p) == C.CRYSTAL_OK
            tasks.append(t)
        got = []
        for t, (st, _) in zip(tasks, want):
            assert t.wait(60_000_000_000) == (C.CRYSTAL_OK if st == 0 else C.CRYSTAL_EOVERFLOW)
            got.append(t.output())
        _compare(jobs, got, want, "runtime")
        for t in tasks:
            t.release()
