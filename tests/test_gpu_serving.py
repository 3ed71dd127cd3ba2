"""The serving loop on the GPU: Poisson arrivals, lognormal sizes, mixed
direct / sliding requests, admission against a small device pool (so
requests wait for room), continuous batching.  Every captured output must be
bit-exact against the oracle, and the same as the request run alone."""
import numpy as np
import pytest

from helpers import first_difference, same_result

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    import torch

    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    from paper_1005_1695_b300 import crystal

    crystal.load()
    return crystal


def _outputs(req, res, capture):
    outs = {}
    for i in range(len(req)):
        off = int(req["capture_offset"][i])
        if off != (1 << 64) - 1:
            outs[i] = capture[off:off + int(res["used_bytes"][i])].tobytes()
    return outs


@pytest.mark.parametrize("pinned,ring", [(False, 0), (True, 0), (True, 2 << 20), (False, 2 << 20)],
                         ids=["staged", "pinned_source", "pinned_ring", "staged_ring"])
def test_served_mix_bit_exact_alone_equals_mix(C, oracle_mod, pinned, ring):
    from paper_1005_1695_b300 import inputs
    from paper_1005_1695_b300 import streams as S

    src = inputs.arena(3, 64 << 20, out=C.page_aligned(64 << 20))
    req, cap = S.make_trace(3, 240, 4000.0, src.nbytes, median=96 << 10, sigma=1.5, cap=4 << 20,
                            capture_every=1)
    # a device pool far smaller than the trace's total bytes: admission has to
    # wait; the 2 MiB input ring (requests up to 256 KiB) wraps many times and
    # is full at times, so some small requests get buffers of their own
    st, res, wall, capture = S.serve_trace(req, src, device_pool_bytes=24 << 20, host_pool_bytes=24 << 20,
                                           streams=4, batch_jobs=4, copy_threads=4, capture_bytes=cap,
                                           source_pinned=pinned, ring_bytes=ring)
    assert st == C.CRYSTAL_OK
    assert (res["status"] == 0).all()
    assert (res["done_ns"] >= res["submit_ns"]).all() and (res["submit_ns"] >= res["admit_ns"]).all()
    assert (res["admit_ns"] >= req["arrival_ns"]).all()
    assert wall > 0
    mix = _outputs(req, res, capture)
    for i in range(len(req)):
        k, n, o = int(req["kind"][i]), int(req["size"][i]), int(req["src_offset"][i])
        ost, want = oracle_mod.task(k, src[o:o + n], int(req["out_size"][i]))
        assert ost == 0
        assert same_result(k, n, mix[i], want), f"request {i}: " + first_difference(k, n, mix[i], want)
    # the same requests one at a time, each alone on the GPU
    for i in range(0, len(req), 12):
        one = req[i:i + 1].copy()
        one["arrival_ns"] = 0
        one["capture_offset"] = 0
        st1, res1, _, cap1 = S.serve_trace(one, src, device_pool_bytes=64 << 20, host_pool_bytes=64 << 20,
                                           streams=1, batch_jobs=1, copy_threads=1,
                                           capture_bytes=int(one["out_size"][0]) + 16)
        assert st1 == C.CRYSTAL_OK
        alone = cap1[:int(res1["used_bytes"][0])].tobytes()
        assert alone == mix[i], i


def test_request_that_never_fits_fails_cleanly(C):
    from paper_1005_1695_b300 import inputs
    from paper_1005_1695_b300 import streams as S

    src = inputs.arena(4, 16 << 20)
    req, _ = S.make_trace(4, 20, 2000.0, src.nbytes, median=64 << 10, cap=1 << 20, p_sliding=0.0)
    req["size"][5] = 12 << 20  # larger than the whole device pool below
    req["src_offset"][5] = 0
    st, res, wall, _ = S.serve_trace(req, src, device_pool_bytes=8 << 20, host_pool_bytes=64 << 20,
                                     streams=2, batch_jobs=2)
    assert res["status"][5] == C.CRYSTAL_ENOMEM
    others = np.delete(res["status"], 5)
    assert (others == 0).all()
    assert st == C.CRYSTAL_ENOMEM


@pytest.mark.parametrize("arrival_order", [False, True], ids=["bypass", "arrival_order"])
def test_admission_past_a_blocked_large_request(C, oracle_mod, arrival_order):
    """Two 12 MiB requests (3 and 5) cannot be resident together in a 20 MiB
    device pool.  While request 5 waits for room, the small requests behind it
    that fit are admitted past it (for a bounded time); with strict arrival
    order nothing passes it.  Every output stays bit-exact either way."""
    from paper_1005_1695_b300 import inputs
    from paper_1005_1695_b300 import streams as S

    src = inputs.arena(6, 32 << 20, out=C.page_aligned(32 << 20))
    req, _ = S.make_trace(6, 40, 1000.0, src.nbytes, median=64 << 10, sigma=0.5, cap=256 << 10, p_sliding=0.3)
    req["arrival_ns"] = 0  # all waiting at once
    for i in (3, 5):
        req["size"][i] = 12 << 20
        req["src_offset"][i] = 1 << 20
        req["kind"][i] = C.CRYSTAL_KIND_MD5_DIRECT
    S.set_out_sizes(req)
    cap = S.assign_capture(req)
    st, res, wall, capture = S.serve_trace(req, src, device_pool_bytes=20 << 20, host_pool_bytes=64 << 20,
                                           streams=4, batch_jobs=4, copy_threads=4, capture_bytes=cap,
                                           source_pinned=True, arrival_order=arrival_order,
                                           bypass_ns=1_000_000_000)
    assert st == C.CRYSTAL_OK and (res["status"] == 0).all()
    admit = res["admit_ns"].astype(np.int64)
    passed = int((admit[6:] < admit[5]).sum())
    if arrival_order:
        assert (np.diff(admit) >= 0).all() and passed == 0
    else:
        assert passed > 0
    for i in range(len(req)):
        k, n, o = int(req["kind"][i]), int(req["size"][i]), int(req["src_offset"][i])
        ost, want = oracle_mod.task(k, src[o:o + n], int(req["out_size"][i]))
        off = int(req["capture_offset"][i])
        got = capture[off:off + int(res["used_bytes"][i])].tobytes()
        assert ost == 0 and same_result(k, n, got, want), f"request {i}: " + first_difference(k, n, got, want)



@pytest.mark.parametrize("pinned", [True, False], ids=["pinned_source", "staged"])
def test_input_ring_merges_small_requests(C, oracle_mod, pinned):
    """64 requests of 40-200 KiB waiting at once, read from scattered offsets
    of the source: through the input ring, requests admitted one after another
    sit side by side in pinned and device memory, and each batch copies its
    ring inputs in one transfer.  Without the ring every request (read in
    place) is its own transfer.  Every output is bit-exact either way."""
    from paper_1005_1695_b300 import inputs
    from paper_1005_1695_b300 import streams as S

    src = inputs.arena(8, 32 << 20, out=C.page_aligned(32 << 20))
    req, _ = S.make_trace(8, 64, 1000.0, src.nbytes, median=96 << 10, sigma=0.4, cap=200 << 10, p_sliding=0.25)
    req["arrival_ns"] = 0
    req["size"] = np.maximum(req["size"], 40 << 10)
    req["src_offset"] = np.minimum(req["src_offset"], src.nbytes - req["size"])
    S.set_out_sizes(req)
    cap = S.assign_capture(req)
    if pinned:
        C.host_register(src)
    copies = {}
    try:
        for ring in (0, 32 << 20):
            ctx = C.Context(max_in_bytes=256 << 10, max_out_bytes=1 << 20, device_pool_bytes=128 << 20,
                            host_pool_bytes=128 << 20, n_streams=2, max_batch_jobs=16,
                            max_batch_bytes=32 << 20, flags=C.CRYSTAL_FLAG_GRAPHS)
            capture = np.zeros(cap, dtype=np.uint8)
            try:
                st, res, _ = ctx.serve(src, req, capture=capture, copy_threads=4, source_pinned=pinned,
                                       ring_bytes=ring)
                copies[ring] = int(ctx.stats().copies_dma)
            finally:
                ctx.shutdown()
            assert st == C.CRYSTAL_OK and (res["status"] == 0).all()
            for i in range(len(req)):
                k, n, o = int(req["kind"][i]), int(req["size"][i]), int(req["src_offset"][i])
                ost, want = oracle_mod.task(k, src[o:o + n], int(req["out_size"][i]))
                off = int(req["capture_offset"][i])
                got = capture[off:off + int(res["used_bytes"][i])].tobytes()
                assert ost == 0 and same_result(k, n, got, want), \
                    f"ring {ring}, request {i}: " + first_difference(k, n, got, want)
    finally:
        if pinned:
            C.host_unregister(src)
    sliding = int(np.isin(req["kind"], list(C.SLIDING_KINDS)).sum())
    if pinned:
        assert copies[0] >= len(req)  # every input in place is its own transfer
    # ring inputs merge: fewer input transfers than requests (outputs of the
    # sliding requests are copied back on their own at most)
    assert copies[32 << 20] - sliding < len(req) // 2, copies


def test_input_ring_larger_than_the_pools_is_refused(C):
    from paper_1005_1695_b300 import inputs
    from paper_1005_1695_b300 import streams as S

    src = inputs.arena(9, 4 << 20)
    req, _ = S.make_trace(9, 8, 1000.0, src.nbytes, median=16 << 10, cap=64 << 10, p_sliding=0.0)
    ctx = C.Context(max_in_bytes=1 << 20, max_out_bytes=1 << 16, device_pool_bytes=16 << 20,
                    host_pool_bytes=16 << 20, n_streams=1)
    try:
        before = ctx.stats()
        st, res, _ = ctx.serve(src, req, ring_bytes=64 << 20)
        assert st in (C.CRYSTAL_EAGAIN, C.CRYSTAL_ENOMEM)
        st, res, _ = ctx.serve(src, req, ring_bytes=1 << 20)
        assert st == C.CRYSTAL_OK and (res["status"] == 0).all()
        after = ctx.stats()  # the ring and every job's buffers are back in the pools
        assert after.device_pool_used == before.device_pool_used
        assert after.host_pool_used == before.host_pool_used
    finally:
        ctx.shutdown()


def test_served_mixed_hashes_through_the_ring(C, oracle_mod):
    """MD5 and SHA-1, direct and sliding, served together with small requests
    through a 4 MiB input ring (so batches mix kinds, ring slots and buffers
    of their own): every output bit-exact against the oracle."""
    from paper_1005_1695_b300 import inputs
    from paper_1005_1695_b300 import streams as S

    src = inputs.arena(12, 48 << 20, out=C.page_aligned(48 << 20))
    req, _ = S.make_trace(12, 200, 5000.0, src.nbytes, median=96 << 10, sigma=1.2, cap=2 << 20, p_sliding=0.4)
    sha = np.arange(len(req)) % 2 == 1
    req["kind"] = np.where(sha, np.where(np.isin(req["kind"], list(C.SLIDING_KINDS)), C.CRYSTAL_KIND_SHA1_SLIDING,
                                         C.CRYSTAL_KIND_SHA1_DIRECT), req["kind"])
    S.set_out_sizes(req)
    cap = S.assign_capture(req)
    st, res, wall, capture = S.serve_trace(req, src, device_pool_bytes=96 << 20, host_pool_bytes=96 << 20,
                                           streams=4, batch_jobs=8, copy_threads=4, capture_bytes=cap,
                                           source_pinned=True, ring_bytes=4 << 20)
    assert st == C.CRYSTAL_OK and (res["status"] == 0).all()
    for i in range(len(req)):
        k, n, o = int(req["kind"][i]), int(req["size"][i]), int(req["src_offset"][i])
        ost, want = oracle_mod.task(k, src[o:o + n], int(req["out_size"][i]))
        off = int(req["capture_offset"][i])
        got = capture[off:off + int(res["used_bytes"][i])].tobytes()
        assert ost == 0 and same_result(k, n, got, want), f"request {i} (kind {k}): " + first_difference(k, n, got, want)
