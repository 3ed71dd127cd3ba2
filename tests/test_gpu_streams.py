"""Job streams in every form the runtime offers (pooled / staged / no overlap /
per-job allocation / plain), bit-exact against the CPU oracle."""
import concurrent.futures as cf
import os

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


MODE_KINDS = [(m, k) for m in ("pooled", "pooled_staged", "no_overlap", "per_job_malloc", "plain") for k in (1, 2)] + \
    [(m, k) for m in ("pooled", "pooled_staged") for k in (3, 4)]


@pytest.mark.parametrize("mode,kind", MODE_KINDS,
                         ids=[f"{m}-{['', 'direct', 'sliding', 'sha1_direct', 'sha1_sliding'][k]}" for m, k in MODE_KINDS])
def test_stream_modes_bit_exact(C, oracle_mod, mode, kind):
    from paper_1005_1695_b300 import inputs
    from paper_1005_1695_b300 import streams as S

    n_units, n = 40, 300_017
    sliding = kind in (2, 4)
    p = C.params(mask=0x3FF, target=0x3FF) if sliding else C.params(segment_bytes=4096)
    out_size = C.sliding_out_bytes(n, n // 256, kind) if sliding else C.digest_size(kind)

    def unit(i):
        return inputs.dedup_unit(5, i, n) if sliding else inputs.uniform_unit(5, i, n)

    r = S.run_stream(mode, unit, n_units, n, kind, p, out_size, streams=3, batch_jobs=4, depth=6,
                     keep=range(n_units))
    assert r.statuses == [C.CRYSTAL_OK] * n_units
    assert len(r.latencies_ms) == n_units and min(r.latencies_ms) >= 0
    checked = list(range(0, n_units, 3))

    def oracle(i):
        return oracle_mod.task(kind, unit(i), out_size, seg_bytes=p.segment_bytes, window=p.window_bytes,
                               mask=p.mask, target=p.target, chunk_seg_bytes=p.chunk_segment_bytes)

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        wants = list(ex.map(oracle, checked))
    for i, (st, want) in zip(checked, wants):
        assert st == 0
        got = r.outputs[i]
        assert same_result(kind, n, got, want), f"{mode} unit {i}: " + first_difference(kind, n, got, want)


def test_staging_ring_arguments_and_pool_limits(C, oracle_mod):
    """crystal_stream_staged: an empty stream, units of every size up to the
    context's limit with a ring smaller than the stream (jobs reused many
    times), a unit above the limit (EINVAL, nothing processed), and a pool too
    small for the ring (EAGAIN, nothing processed)."""
    from paper_1005_1695_b300 import inputs

    with C.Context(max_in_bytes=1 << 20, max_out_bytes=1 << 16, device_pool_bytes=64 << 20,
                   host_pool_bytes=64 << 20, n_streams=2, max_batch_jobs=4) as ctx:
        st, res, wall, outs = ctx.stream_staged([], C.CRYSTAL_KIND_MD5_DIRECT, 16)
        assert st == C.CRYSTAL_OK and len(res) == 0
        sizes = [0, 1, 63, 64, 4095, 4096, 4097, 100_003, 1 << 20] * 3
        units = [inputs.uniform_unit(61, i, n) for i, n in enumerate(sizes)]
        st, res, wall, outs = ctx.stream_staged(units, C.CRYSTAL_KIND_MD5_DIRECT, 16, C.params(), copy_threads=3,
                                                ring_jobs=4)
        assert st == C.CRYSTAL_OK and (res["status"] == 0).all() and wall > 0
        assert (res["used_bytes"] == 16).all()
        for i, u in enumerate(units):
            assert outs[i, :16].tobytes() == oracle_mod.direct(u, 4096), i
        too_big = [np.zeros((1 << 20) + 1, dtype=np.uint8)]
        st, res, _, _ = ctx.stream_staged(too_big, C.CRYSTAL_KIND_MD5_DIRECT, 16)
        assert st == C.CRYSTAL_EINVAL and res["status"][0] == 0 and res["done_ns"][0] == 0
        # 100 ring jobs of 1 MiB do not fit a 64 MiB pool
        big = [np.zeros(1 << 20, dtype=np.uint8)] * 100
        st, res, _, _ = ctx.stream_staged(big, C.CRYSTAL_KIND_MD5_DIRECT, 16, ring_jobs=100)
        assert st in (C.CRYSTAL_EAGAIN, C.CRYSTAL_ENOMEM) and (res["done_ns"] == 0).all()
        assert ctx.stats().device_pool_used < (1 << 20)  # the partial ring was given back
