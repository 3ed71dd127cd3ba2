"""Each of the five workload configurations at its stated shape, through the
form the benchmark runs it in, every unit bit-exact against the CPU oracle.

* 1  plain direct hashing, 64 x 64 KiB, 4 KiB segments, one stream, one job
     at a time (and the pooled form of the same units);
* 2  sliding-window hashing, 256 x 1 MiB (half repeated 8 KiB blocks), w = 20,
     mask = target = 0x1FFF, chunk direct hash S = 4 KiB: device-resident
     launches and the job API with graphs, 8 streams x 8 jobs;
* 3  pipelined direct hashing of 4 MiB units, pooled buffers over 8 streams
     (resident jobs and the staged ring from pageable memory);
* 4  uneven batches: log-uniform 4 KiB - 16 MiB (several units at the 16 MiB
     cap), 80/20 direct/sliding, read in place from a page-locked arena,
     autotuned, replayed as CUDA graphs;
* 5  served Poisson stream: lognormal sizes (median 256 KiB, sigma 1.5, cap
     64 MiB) with two requests at the cap, 70/30 direct/sliding, admission
     against a device pool too small for both capped requests at once; every
     request also equals the same request served alone.

The paper measures these shapes as streams of data blocks (Section 5.2,
Figures 6-8); the sizes are the configurations' own.
"""
import concurrent.futures as cf
import os

import numpy as np
import pytest

from helpers import first_difference, same_result

pytestmark = pytest.mark.gpu

DIRECT, SLIDING = 1, 2
SEC = 1_000_000_000
THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module")
def C():
    import torch

    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    from paper_1005_1695_b300 import crystal

    crystal.load()
    return crystal


def _oracle_many(oracle_mod, jobs):
    """jobs: (kind, bytes-like, out_size, params-or-None); returns (status, out)."""

    def one(j):
        kind, data, out_size, p = j
        kw = {} if p is None else dict(seg_bytes=p.segment_bytes, window=p.window_bytes, mask=p.mask,
                                        target=p.target, chunk_seg_bytes=p.chunk_segment_bytes)
        return oracle_mod.task(kind, data, out_size, **kw)

    # the largest jobs first, so the longest oracle calls start at once
    order = sorted(range(len(jobs)), key=lambda i: -len(jobs[i][1]))
    out = [None] * len(jobs)
    with cf.ThreadPoolExecutor(max_workers=THREADS) as ex:
        for i, r in zip(order, ex.map(one, [jobs[i] for i in order])):
            out[i] = r
    return out


def _assert_same(kind, n, got, want, what):
    assert same_result(kind, n, got, want), f"{what}: " + first_difference(kind, n, got, want)


# ---- configuration 1 ---------------------------------------------------------------

@pytest.mark.parametrize("mode", ["plain", "pooled"])
def test_config1_plain_direct_64x64k_every_unit(C, oracle_mod, mode):
    from paper_1005_1695_b300 import inputs
    from paper_1005_1695_b300 import streams as S

    U, N = 64, 65536
    p = C.params(segment_bytes=4096)
    units = [inputs.uniform_unit(1, i, N) for i in range(U)]
    r = S.run_stream(mode, lambda i: units[i], U, N, DIRECT, p, 16, streams=8, batch_jobs=8, keep=range(U))
    assert r.statuses == [C.CRYSTAL_OK] * U
    want = _oracle_many(oracle_mod, [(DIRECT, u, 16, p) for u in units])
    for i in range(U):
        assert want[i][0] == 0
        _assert_same(DIRECT, N, r.outputs[i], want[i][1], f"{mode} unit {i}")


# ---- configuration 2 ---------------------------------------------------------------

@pytest.fixture(scope="module")
def config2(C, oracle_mod):
    """The 256 x 1 MiB sliding workload with the oracle's output for every unit."""
    from paper_1005_1695_b300 import inputs

    U, N = 256, 1 << 20
    pool = inputs.dedup_pool(2)
    host = np.empty(U * N, dtype=np.uint8)
    for u in range(U):
        inputs.dedup_unit(2, u, N, pool=pool, out=host[u * N:(u + 1) * N])
    p = C.params(window_bytes=20, mask=0x1FFF, target=0x1FFF, chunk_segment_bytes=4096)
    out_size = C.sliding_out_bytes(N, 1024)
    want = _oracle_many(oracle_mod, [(SLIDING, host[u * N:(u + 1) * N], out_size, p) for u in range(U)])
    assert all(st == 0 for st, _ in want)
    return host, U, N, p, out_size, want


def test_config2_device_resident_every_unit(C, config2):
    """The launch sequence the benchmark times for `value`: one 256-unit batch
    on a device-resident descriptor, window / chunk / digest launches."""
    import torch

    host, U, N, p, out_size, want = config2
    d_in = torch.from_numpy(host).cuda()
    b = C.DeviceBatch(d_in, [u * N for u in range(U)], [N] * U, [SLIDING] * U, p, out_sizes=[out_size] * U)
    for _ in range(2):  # the benchmark replays the same descriptor step after step
        b.d_desc.copy_(torch.from_numpy(b.host_desc).cuda())
        b.launch_sliding_windows()
        b.launch_sliding_chunks()
        b.launch_sliding_digests()
        torch.cuda.synchronize()
        assert b.device_status() == 0
        got = b.outputs()
        for u in range(U):
            _assert_same(SLIDING, N, got[u], want[u][1], f"unit {u}")


def test_config2_job_api_every_unit(C, config2):
    """The end-to-end form: pooled pinned jobs, 8 streams, 8 jobs per batch,
    CUDA graphs, all 256 submitted at once (as the benchmark's e2e leg)."""
    from paper_1005_1695_b300 import streams as S

    host, U, N, p, out_size, want = config2
    r = S.run_stream("pooled", lambda i: host[i * N:(i + 1) * N], U, N, SLIDING, p, out_size, streams=8,
                     batch_jobs=8, graphs=True, keep=range(U))
    assert r.statuses == [C.CRYSTAL_OK] * U
    for u in range(U):
        _assert_same(SLIDING, N, r.outputs[u], want[u][1], f"unit {u}")


# ---- configuration 3 ---------------------------------------------------------------

@pytest.fixture(scope="module")
def config3(C, oracle_mod):
    from paper_1005_1695_b300 import inputs

    U, N = 256, 4 << 20
    units = [inputs.uniform_unit(3, i, N) for i in range(U)]
    p = C.params(segment_bytes=4096)
    want = _oracle_many(oracle_mod, [(DIRECT, u, 16, p) for u in units])
    return units, U, N, p, want


@pytest.mark.parametrize("mode", ["pooled", "pooled_staged"])
def test_config3_pipelined_4mib_every_unit(C, config3, mode):
    """256 units of 4 MiB (1 GiB) through the pooled, overlapped runtime: jobs
    resident in pinned buffers, and the staged ring fed from pageable memory by
    copy threads."""
    from paper_1005_1695_b300 import streams as S

    units, U, N, p, want = config3
    r = S.run_stream(mode, lambda i: units[i], U, N, DIRECT, p, 16, streams=8, batch_jobs=8, depth=48,
                     keep=range(U))
    assert r.statuses == [C.CRYSTAL_OK] * U
    for u in range(U):
        _assert_same(DIRECT, N, r.outputs[u], want[u][1], f"{mode} unit {u}")


# ---- configuration 4 ---------------------------------------------------------------

def test_config4_uneven_full_size_range_every_unit(C, oracle_mod):
    """1,000 units drawn log-uniform over the whole 4 KiB - 16 MiB range, four
    of them (two direct, two sliding) at the 16 MiB cap, 80/20 direct/sliding,
    read in place from a page-locked arena, packed into batches replayed as CUDA
    graphs with the setting the autotuner picks."""
    from paper_1005_1695_b300 import autotune as A
    from paper_1005_1695_b300 import inputs
    from paper_1005_1695_b300 import streams as S

    arena_bytes = 256 << 20
    src = inputs.arena(41, arena_bytes, out=C.page_aligned(arena_bytes))
    req, _ = S.make_batch(41, 1000, src.nbytes, lo=4096, hi=16 << 20)
    assert req["size"].min() >= 4096 and req["size"].max() <= 16 << 20
    for k, i in enumerate((3, 250, 500, 750)):
        req["size"][i] = 16 << 20
        req["src_offset"][i] = (k * (48 << 20)) + 7 * k
        req["kind"][i] = DIRECT if k < 2 else SLIDING
    S.set_out_sizes(req)
    cap = S.assign_capture(req)
    C.host_register(src)
    try:
        best, table = A.tune(req[:300], src, device_pool_bytes=1 << 30, streams=(4, 8), batch_jobs=(8, 32),
                             batch_bytes=(64 << 20,), ring_max=(0, 256 << 10), repeats=1)
        capture = np.zeros(cap, dtype=np.uint8)
        st, res, wall = A.run_batch(req, src, best, device_pool_bytes=1 << 30, capture=capture)
    finally:
        C.host_unregister(src)
    assert st == C.CRYSTAL_OK and (res["status"] == 0).all()
    jobs = [(int(r["kind"]), src[int(r["src_offset"]):int(r["src_offset"]) + int(r["size"])], int(r["out_size"]),
             None) for r in req]
    want = _oracle_many(oracle_mod, jobs)
    for i, r in enumerate(req):
        k, n, off = int(r["kind"]), int(r["size"]), int(r["capture_offset"])
        assert want[i][0] == 0
        got = capture[off:off + int(res["used_bytes"][i])].tobytes()
        _assert_same(k, n, got, want[i][1], f"unit {i} ({n} B, kind {k})")


# ---- configuration 5 ---------------------------------------------------------------

@pytest.fixture(scope="module")
def config5(C, oracle_mod):
    from paper_1005_1695_b300 import inputs
    from paper_1005_1695_b300 import streams as S

    src_bytes = 160 << 20
    src = inputs.arena(51, src_bytes, out=C.page_aligned(src_bytes))
    req, _ = S.make_trace(51, 300, 4000.0, src.nbytes, median=256 << 10, sigma=1.5, cap=64 << 20)
    big = (120, 126)  # two requests at the cap, close together in arrival order
    for k, i in enumerate(big):
        req["size"][i] = 64 << 20
        req["src_offset"][i] = k * (80 << 20) + 3
        req["kind"][i] = DIRECT if k == 0 else SLIDING
    S.set_out_sizes(req)
    S.assign_capture(req)
    jobs = [(int(r["kind"]), src[int(r["src_offset"]):int(r["src_offset"]) + int(r["size"])], int(r["out_size"]),
             None) for r in req]
    want = _oracle_many(oracle_mod, jobs)
    assert all(st == 0 for st, _ in want)
    return src, req, big, want


@pytest.mark.parametrize("pinned,ring", [(True, 0), (False, 0), (True, 64 << 20)],
                         ids=["pinned_source", "staged", "pinned_ring"])
def test_config5_served_lognormal_with_capped_requests(C, config5, pinned, ring):
    from paper_1005_1695_b300 import streams as S

    src, req, big, want = config5
    cap = int(req["capture_offset"].max() + req["out_size"][np.argmax(req["capture_offset"])]) + 16
    # 96 MiB of device pool: the capped sliding request alone takes about 73 MiB,
    # so the two capped requests can never be resident together
    pool = 96 << 20
    assert C.scratch_bytes(SLIDING, 64 << 20, int(req["out_size"][big[1]])) + (64 << 20) + \
        int(req["out_size"][big[1]]) + (64 << 20) > pool
    # with the 64 MiB input ring (requests up to 256 KiB) the pool holds the
    # ring beside the capped requests' buffers
    st, res, wall, capture = S.serve_trace(req, src, device_pool_bytes=pool + ring, host_pool_bytes=pool + ring,
                                           streams=8, batch_jobs=8, copy_threads=4, capture_bytes=cap,
                                           source_pinned=pinned, ring_bytes=ring)
    assert st == C.CRYSTAL_OK and (res["status"] == 0).all()
    assert (res["admit_ns"] >= req["arrival_ns"]).all() and (res["done_ns"] >= res["submit_ns"]).all()
    mix = {}
    for i in range(len(req)):
        k, n, off = int(req["kind"][i]), int(req["size"][i]), int(req["capture_offset"][i])
        mix[i] = capture[off:off + int(res["used_bytes"][i])].tobytes()
        _assert_same(k, n, mix[i], want[i][1], f"request {i} ({n} B, kind {k})")
    # alone == in the mix: every 10th request and both capped ones, each served alone
    for i in sorted(set(range(0, len(req), 10)) | set(big)):
        one = req[i:i + 1].copy()
        one["arrival_ns"] = 0
        one["capture_offset"] = 0
        st1, res1, _, cap1 = S.serve_trace(one, src, device_pool_bytes=pool, host_pool_bytes=pool, streams=1,
                                           batch_jobs=1, copy_threads=1, capture_bytes=int(one["out_size"][0]) + 16,
                                           source_pinned=pinned)
        assert st1 == C.CRYSTAL_OK
        assert cap1[:int(res1["used_bytes"][0])].tobytes() == mix[i], i


# ---- the headline workload with SHA-1 (the hash of the paper's own runs) ----------

def test_config2_sha1_every_unit(C, oracle_mod):
    """Configuration 2's 256 x 1 MiB units hashed with SHA-1 (Section 5.2's hash):
    the device-resident launches the benchmark times, every unit against the
    oracle."""
    import torch

    from paper_1005_1695_b300 import inputs

    U, N = 256, 1 << 20
    SHA1_SLIDING = C.CRYSTAL_KIND_SHA1_SLIDING
    pool = inputs.dedup_pool(2)
    host = np.empty(U * N, dtype=np.uint8)
    for u in range(U):
        inputs.dedup_unit(2, u, N, pool=pool, out=host[u * N:(u + 1) * N])
    p = C.params(window_bytes=20, mask=0x1FFF, target=0x1FFF, chunk_segment_bytes=4096)
    out_size = C.sliding_out_bytes(N, 1024, SHA1_SLIDING)
    d_in = torch.from_numpy(host).cuda()
    b = C.DeviceBatch(d_in, [u * N for u in range(U)], [N] * U, [SHA1_SLIDING] * U, p, out_sizes=[out_size] * U)
    b.launch_sliding_windows()
    b.launch_sliding_chunks()
    b.launch_sliding_digests()
    torch.cuda.synchronize()
    assert b.device_status() == 0
    got = b.outputs()
    want = _oracle_many(oracle_mod, [(SHA1_SLIDING, host[u * N:(u + 1) * N], out_size, p) for u in range(U)])
    for u in range(U):
        assert want[u][0] == 0
        _assert_same(SHA1_SLIDING, N, got[u], want[u][1], f"unit {u}")
