"""crystal_md5_direct_noalloc: direct hashing for callers that cannot allocate
device memory where they hash (a latency-bound storage or network data path,
where cudaMalloc/cudaFree could synchronise the device, or a process whose
free device memory belongs to another allocator).  Its scratch is a fixed
array inside the library; this checks, through the C ABI, that two calls in a
row give the same digests as the allocating batch launcher and as the CPU
oracle, that a request exactly at the array's size is accepted and correct,
and that one unit or one segment more is refused.

This file is collected last on purpose, so that a run stopping at the first
failure has run every other test first.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

DIRECT = 1
SCRATCH_BYTES = 8 << 20  # CRYSTAL_NOALLOC_SCRATCH_BYTES


@pytest.fixture(scope="module")
def env():
    import torch

    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    from paper_1005_1695_b300 import crystal

    lib = crystal.load()
    fn = lib.crystal_md5_direct_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p,
                   ctypes.c_void_p]
    return torch, crystal, fn


def _reference(torch, C, d_in, unit_bytes, n_units, seg):
    """Digests from the existing entry point (caller-allocated scratch)."""
    b = C.DeviceBatch(d_in, [u * unit_bytes for u in range(n_units)], [unit_bytes] * n_units,
                      [DIRECT] * n_units, C.params(segment_bytes=seg))
    b.launch_direct()
    torch.cuda.synchronize()
    return [o[:16] for o in b.outputs()]


def _noalloc(torch, fn, d_in, unit_bytes, n_units, seg):
    out = torch.full((16 * n_units,), 0xAB, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    st = fn(d_in.data_ptr(), unit_bytes, n_units, seg, out.data_ptr(), stream)
    assert st == 0, st
    torch.cuda.synchronize()
    host = out.cpu().numpy()
    return [host[16 * u:16 * (u + 1)].tobytes() for u in range(n_units)]


def test_noalloc_matches_existing_entry_point_twice(env, oracle_mod):
    torch, C, fn = env
    from paper_1005_1695_b300 import inputs

    cases = [(65536, 64, 4096), (100003, 37, 1000)]  # second call: other sizes, ragged tails
    for unit_bytes, n_units, seg in cases:
        host = np.concatenate([inputs.uniform_unit(31, u, unit_bytes) for u in range(n_units)])
        d_in = torch.from_numpy(host).cuda()
        want = _reference(torch, C, d_in, unit_bytes, n_units, seg)
        got = _noalloc(torch, fn, d_in, unit_bytes, n_units, seg)
        assert got == want, (unit_bytes, n_units, seg)
        oracle = [oracle_mod.direct(host[u * unit_bytes:(u + 1) * unit_bytes], seg) for u in range(n_units)]
        assert got == oracle, (unit_bytes, n_units, seg)


def _limit_case():
    """16 units of 32,763 segments of 64 bytes: align_up(64 + 64 * 16, 256) +
    16 * 16 * 32,763 = 1,280 + 8,387,328 bytes, exactly the array's size."""
    n_units, seg, m = 16, 64, 32763
    desc = (64 + 64 * n_units + 255) // 256 * 256
    assert desc + 16 * n_units * m == SCRATCH_BYTES
    return n_units, seg, m * seg


def test_noalloc_exactly_at_the_limit(env, oracle_mod):
    torch, C, fn = env
    from paper_1005_1695_b300 import inputs

    n_units, seg, unit_bytes = _limit_case()
    host = np.concatenate([inputs.uniform_unit(32, u, unit_bytes) for u in range(n_units)])
    d_in = torch.from_numpy(host).cuda()
    got = _noalloc(torch, fn, d_in, unit_bytes, n_units, seg)
    want = [oracle_mod.direct(host[u * unit_bytes:(u + 1) * unit_bytes], seg) for u in range(n_units)]
    assert got == want


def test_noalloc_refuses_requests_above_the_array(env):
    torch, C, fn = env
    n_units, seg, unit_bytes = _limit_case()
    d_in = torch.zeros((n_units + 1) * unit_bytes + 1, dtype=torch.uint8, device="cuda")
    out = torch.zeros(16 * 4096, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    # one unit more, or one byte more per unit (one more segment each), than the limit
    assert fn(d_in.data_ptr(), unit_bytes, n_units + 1, seg, out.data_ptr(), stream) == C.CRYSTAL_EINVAL
    assert fn(d_in.data_ptr(), unit_bytes + 1, n_units, seg, out.data_ptr(), stream) == C.CRYSTAL_EINVAL
    # 4096 units of 1 MiB at 1 KiB segments need 64 MiB of digests
    assert fn(d_in.data_ptr(), 1 << 20, 4096, 1024, out.data_ptr(), stream) == C.CRYSTAL_EINVAL
    assert fn(d_in.data_ptr(), 1 << 20, 1, 0, out.data_ptr(), stream) == C.CRYSTAL_EINVAL
    assert fn(None, 1 << 20, 1, 4096, out.data_ptr(), stream) == C.CRYSTAL_EINVAL
