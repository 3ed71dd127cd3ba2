"""Job streams in every form the runtime offers (pooled / staged / no overlap /
per-job allocation / plain), bit-exact against the CPU oracle."""
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


@pytest.mark.parametrize("mode", ["pooled", "pooled_staged", "no_overlap", "per_job_malloc", "plain"])
@pytest.mark.parametrize("kind", [1, 2], ids=["direct", "sliding"])
def test_stream_modes_bit_exact(C, oracle_mod, mode, kind):
    from paper_1005_1695_b300 import inputs
    from paper_1005_1695_b300 import streams as S

    n_units, n = 40, 300_017
    p = C.params(mask=0x3FF, target=0x3FF) if kind == 2 else C.params(segment_bytes=4096)
    out_size = 16 if kind == 1 else C.sliding_out_bytes(n, n // 256)

    def unit(i):
        return inputs.dedup_unit(5, i, n) if kind == 2 else inputs.uniform_unit(5, i, n)

    r = S.run_stream(mode, unit, n_units, n, kind, p, out_size, streams=3, batch_jobs=4, depth=6,
                     keep=range(n_units))
    assert r.statuses == [C.CRYSTAL_OK] * n_units
    assert len(r.latencies_ms) == n_units and min(r.latencies_ms) >= 0
    for i in range(0, n_units, 3):
        st, want = oracle_mod.task(kind, unit(i), out_size, seg_bytes=p.segment_bytes, window=p.window_bytes,
                                   mask=p.mask, target=p.target, chunk_seg_bytes=p.chunk_segment_bytes)
        assert st == 0
        got = r.outputs[i]
        assert same_result(kind, n, got, want), f"{mode} unit {i}: " + first_difference(kind, n, got, want)
