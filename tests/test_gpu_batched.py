"""Batches of uneven units (log-uniform sizes, mixed direct / sliding) read in
place from a page-locked arena, replayed as CUDA graphs, with the setting
the autotuner picks: every unit bit-exact against the oracle."""
import concurrent.futures as cf
import os

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


def test_batched_uneven_autotuned_bit_exact(C, oracle_mod):
    from paper_1005_1695_b300 import autotune as A
    from paper_1005_1695_b300 import inputs
    from paper_1005_1695_b300 import streams as S

    src = inputs.arena(8, 128 << 20, out=C.page_aligned(128 << 20))
    req, cap = S.make_batch(8, 1200, src.nbytes, lo=4096, hi=1 << 20, capture=True)
    C.host_register(src)
    try:
        best, table = A.tune(req[:400], src, device_pool_bytes=512 << 20, streams=(2, 8), batch_jobs=(4, 64),
                             batch_bytes=(32 << 20,), ring_max=(0, 256 << 10), repeats=1)
        assert len(table) == 8 and best.streams in (2, 8) and best.ring_max in (0, 256 << 10)
        best, gtable = A.tune_geometry(req[:400], src, best, device_pool_bytes=512 << 20, repeats=1,
                                       knobs=(("seg_threads", (128, 64)), ("win_ctas_per_sm", (0, 2))))
        assert set(best.geometry) <= {0, 1, 2} and len(best.geometry) >= 2 and len(gtable) >= 2 * len(best.geometry)
        import numpy as np

        # the whole batch with the units up to 256 KiB going through the input ring
        best.ring_max = 256 << 10
        capture = np.zeros(cap, dtype=np.uint8)
        st, res, wall = A.run_batch(req, src, best, device_pool_bytes=512 << 20, capture=capture)
    finally:
        C.host_unregister(src)
    assert st == C.CRYSTAL_OK and (res["status"] == 0).all()

    def check(i):
        k, n, o = int(req["kind"][i]), int(req["size"][i]), int(req["src_offset"][i])
        ost, want = oracle_mod.task(k, src[o:o + n], int(req["out_size"][i]))
        off = int(req["capture_offset"][i])
        got = capture[off:off + int(res["used_bytes"][i])].tobytes()
        return i, ost == 0 and same_result(k, n, got, want), (k, n, got, want)

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        for i, ok, (k, n, got, want) in ex.map(check, range(len(req))):
            assert ok, f"unit {i}: " + first_difference(k, n, got, want)
