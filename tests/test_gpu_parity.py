"""GPU kernels against the CPU oracle, element by element, through the C ABI.

Every output is integer/byte work, so the bar is bit-exact equality of every
result byte (digests, bitmap words, chunk ends, header counts).  Sizes span
several window tiles and segments with ragged tails, odd alignments, the
empty unit, units shorter than the window, every padding branch of MD5, and
the degenerate masks (mask 0 marks every window).
"""
import concurrent.futures as cf
import os

import numpy as np
import pytest

from helpers import first_difference, same_result

pytestmark = pytest.mark.gpu

DIRECT, SLIDING = 1, 2


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return torch


@pytest.fixture(scope="module")
def C():
    from paper_1005_1695_b300 import crystal

    crystal.load()
    return crystal


def _pack(torch, units, align_offsets=None):
    """Place byte arrays in one device buffer at the given misalignments."""
    offs, pos = [], 0
    for i, u in enumerate(units):
        mis = align_offsets[i % len(align_offsets)] if align_offsets else 0
        pos = (pos + 255) // 256 * 256 + mis
        offs.append(pos)
        pos += len(u)
    host = np.zeros(pos + 256, dtype=np.uint8)
    for o, u in zip(offs, units):
        host[o:o + len(u)] = np.frombuffer(bytes(u), dtype=np.uint8) if not isinstance(u, np.ndarray) else u
    return torch.from_numpy(host).cuda(), offs


def _run(torch, C, units, kinds, plist, out_sizes=None, align=None, mode="batch", out_misalign=None):
    d_in, offs = _pack(torch, units, align)
    b = C.DeviceBatch(d_in, offs, [len(u) for u in units], kinds, out_sizes=out_sizes, per_unit_params=plist,
                      out_misalign=out_misalign)
    if mode == "batch":
        b.launch()
    else:
        b.launch_direct_segments()
        b.launch_direct_outer()
        b.launch_sliding_windows()
        b.launch_sliding_chunks()
        b.launch_sliding_digests()
    torch.cuda.synchronize()
    assert b.device_status() == 0
    return b.outputs()


SHA1_DIRECT, SHA1_SLIDING = 3, 4


def _oracle_all(oracle_mod, units, kinds, plist, out_sizes):
    def one(i):
        p = plist[i]
        return oracle_mod.task(kinds[i], bytes(units[i]), out_sizes[i], seg_bytes=p.segment_bytes,
                               window=p.window_bytes, mask=p.mask, target=p.target,
                               chunk_seg_bytes=p.chunk_segment_bytes)

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        return list(ex.map(one, range(len(units))))


def _compare(units, kinds, got, want):
    for i, (g, (st, w)) in enumerate(zip(got, want)):
        assert st in (0, 1)
        assert same_result(kinds[i], len(units[i]), g, w), \
            f"unit {i} n={len(units[i])}: " + first_difference(kinds[i], len(units[i]), g, w)


def _rand(seed, n):
    from paper_1005_1695_b300 import inputs

    return inputs.uniform_unit(seed, 99, n)


# ---- direct hashing -------------------------------------------------------------

DIRECT_SIZES = [0, 1, 3, 55, 56, 57, 63, 64, 65, 119, 120, 127, 128, 4095, 4096, 4097, 8191, 65536, 100003]


@pytest.mark.parametrize("S", [4096, 64, 100, 1, 65536])
def test_direct_sizes_alignments(torch_cuda, C, oracle_mod, S):
    units = [_rand(1000 + i, n) for i, n in enumerate(DIRECT_SIZES)]
    kinds = [DIRECT] * len(units)
    plist = [C.params(segment_bytes=S)] * len(units)
    got = _run(torch_cuda, C, units, kinds, plist, align=[0, 1, 2, 3, 5, 16, 4, 8])
    want = _oracle_all(oracle_mod, units, kinds, plist, [16] * len(units))
    _compare(units, kinds, got, want)


def test_direct_config_64x64k(torch_cuda, C, oracle_mod):
    """64 units of 64 KiB uniform random bytes, 4 KiB segments: every digest."""
    from paper_1005_1695_b300 import inputs

    units = [inputs.uniform_unit(1, i, 65536) for i in range(64)]
    kinds = [DIRECT] * 64
    plist = [C.params()] * 64
    got = _run(torch_cuda, C, units, kinds, plist, mode="split")
    for i, u in enumerate(units):
        assert got[i][:16] == oracle_mod.direct(u, 4096), i


# ---- sliding-window hashing ------------------------------------------------------

@pytest.mark.parametrize("w", [1, 2, 3, 20])
@pytest.mark.parametrize("mask,target", [(0x0, 0x0), (0x1, 0x1), (0x3, 0x0), (0x1FFF, 0x1FFF)])
def test_sliding_tiny_every_length(torch_cuda, C, oracle_mod, w, mask, target):
    units = [_rand(2000 + n, n) for n in range(0, 65)]
    kinds = [SLIDING] * len(units)
    plist = [C.params(window_bytes=w, mask=mask, target=target, chunk_segment_bytes=16)] * len(units)
    outs = [C.out_bytes(SLIDING, len(u), plist[0]) for u in units]
    got = _run(torch_cuda, C, units, kinds, plist, out_sizes=outs, align=[0, 3, 1, 2])
    want = _oracle_all(oracle_mod, units, kinds, plist, outs)
    _compare(units, kinds, got, want)


@pytest.mark.parametrize("w", [20, 7, 16, 55])
@pytest.mark.parametrize("S", [4096, 100])
def test_sliding_ragged_tiles(torch_cuda, C, oracle_mod, w, S):
    sizes = [1023, 1024, 1025, 2047, 2048 + 19, 3000, 10007, 65536 + 5]
    units = [_rand(3000 + i, n) for i, n in enumerate(sizes)]
    kinds = [SLIDING] * len(units)
    plist = [C.params(window_bytes=w, mask=0x3F, target=0x15, chunk_segment_bytes=S)] * len(units)
    outs = [C.sliding_out_bytes(n, n // 16 + 8) for n in sizes]
    got = _run(torch_cuda, C, units, kinds, plist, out_sizes=outs, align=[0, 1, 2, 3, 7, 13])
    want = _oracle_all(oracle_mod, units, kinds, plist, outs)
    _compare(units, kinds, got, want)


@pytest.mark.parametrize("hash_kind", [SLIDING, 4])
def test_sliding_output_alignments_dense_cuts(torch_cuda, C, oracle_mod, hash_kind):
    # outputs at every 4-byte alignment mod 16 (the bitmap scan picks its load
    # width from it); units long enough that each of the chunk kernel's warps
    # walks several iterations of bitmap words, and a mask with many cuts per
    # bitmap word so cut positions interleave across lanes and vectors
    sizes = [300000, 262144 + 4096 * 3 + 5, 1 << 20, 40000, 17]
    units = [_rand(7000 + i, n) for i, n in enumerate(sizes)]
    kinds = [hash_kind] * len(units)
    plist = [C.params(window_bytes=20, mask=0x3F, target=0x2A, chunk_segment_bytes=1000)] * len(units)
    outs = [C.sliding_out_bytes(n, n // 32 + 8, hash_kind) for n in sizes]
    got = _run(torch_cuda, C, units, kinds, plist, out_sizes=outs, align=[0, 5, 11, 2, 8], out_misalign=[4, 8, 12, 0])
    want = _oracle_all(oracle_mod, units, kinds, plist, outs)
    assert all(st == 0 for st, _ in want)
    _compare(units, kinds, got, want)


def test_sliding_overflow_keeps_count(torch_cuda, C, oracle_mod):
    n = 20000
    units = [_rand(5, n)]
    p = C.params(mask=0x7, target=0x7)
    kinds = [SLIDING]
    want = _oracle_all(oracle_mod, units, kinds, [p], [C.sliding_out_bytes(n, n)])
    need = int.from_bytes(want[0][1][:4], "little")
    outs = [C.sliding_out_bytes(n, need - 1)]
    got = _run(torch_cuda, C, units, kinds, [p], out_sizes=outs)
    want = _oracle_all(oracle_mod, units, kinds, [p], outs)
    assert want[0][0] == 1
    _compare(units, kinds, got, want)
    assert int.from_bytes(got[0][4:8], "little") == 1


def test_mixed_batch_params_per_unit(torch_cuda, C, oracle_mod):
    units, kinds, plist, outs = [], [], [], []
    for i in range(24):
        n = [0, 17, 5000, 70000, 1 << 20][i % 5] + i
        units.append(_rand(4000 + i, n))
        if i % 3 == 0:
            kinds.append(SLIDING)
            p = C.params(window_bytes=[20, 12, 33][(i // 3) % 3], mask=0xFF, target=i & 0xFF,
                         chunk_segment_bytes=[4096, 512][i % 2])
            outs.append(C.sliding_out_bytes(n, n // 64 + 4))
        else:
            kinds.append(DIRECT)
            p = C.params(segment_bytes=[4096, 1000, 64][i % 3])
            outs.append(16)
        plist.append(p)
    got = _run(torch_cuda, C, units, kinds, plist, out_sizes=outs, align=[0, 1, 16, 3])
    want = _oracle_all(oracle_mod, units, kinds, plist, outs)
    _compare(units, kinds, got, want)


def test_device_status_word_flags_a_bad_record(torch_cuda, C, oracle_mod):
    """A descriptor edited after crystal_batch_plan so that one sliding unit's
    out_cap is below its fixed header + bitmap: the chunk kernel must skip that
    record and set bit 0 of the batch's device status word (the runtime turns a
    nonzero word into CRYSTAL_EDEVICE), and every other unit must still be
    bit-exact.  The unit's real output buffer is full size, so the window
    kernel's bitmap writes stay inside memory the batch owns: a skip path,
    not a fault."""
    torch = torch_cuda
    sizes = [70001, 200003, 4097]
    units = [_rand(9300 + i, n) for i, n in enumerate(sizes)]
    kinds = [SLIDING] * 3
    p = C.params(mask=0xFF, target=0x11)
    plist = [p] * 3
    outs = [C.sliding_out_bytes(n, n // 64 + 8) for n in sizes]
    d_in, offs = _pack(torch, units, [0, 5, 9])
    b = C.DeviceBatch(d_in, offs, sizes, kinds, out_sizes=outs, per_unit_params=plist)
    recs = b.host_desc[C.BATCH_HEADER_BYTES:].view(C.UNIT_DTYPE)
    bad = [k for k in range(3) if int(recs[k]["in"]) == d_in.data_ptr() + offs[1]]
    assert len(bad) == 1
    fixed = 8 + 4 * ((sizes[1] + 31) // 32)
    recs[bad[0]]["out_cap"] = fixed - 4
    b.d_desc.copy_(torch.from_numpy(b.host_desc).cuda())
    b.launch()
    torch.cuda.synchronize()
    assert b.device_status() & 1
    got = b.outputs()
    want = _oracle_all(oracle_mod, units, kinds, plist, outs)
    keep = [0, 2]
    _compare([units[i] for i in keep], [kinds[i] for i in keep], [got[i] for i in keep], [want[i] for i in keep])


# ---- SHA-1 kinds ------------------------------------------------------------------

@pytest.mark.parametrize("S", [4096, 100, 1])
def test_sha1_direct_sizes_alignments(torch_cuda, C, oracle_mod, S):
    units = [_rand(7000 + i, n) for i, n in enumerate(DIRECT_SIZES)]
    kinds = [SHA1_DIRECT] * len(units)
    plist = [C.params(segment_bytes=S)] * len(units)
    got = _run(torch_cuda, C, units, kinds, plist, align=[0, 1, 2, 3, 5, 16, 4, 8])
    want = _oracle_all(oracle_mod, units, kinds, plist, [20] * len(units))
    _compare(units, kinds, got, want)


@pytest.mark.parametrize("w", [1, 3, 20, 55])
@pytest.mark.parametrize("mask,target", [(0x0, 0x0), (0x3, 0x1), (0x1FFF, 0x1FFF)])
def test_sha1_sliding_tiny_every_length(torch_cuda, C, oracle_mod, w, mask, target):
    units = [_rand(8000 + n, n) for n in range(0, 65)]
    kinds = [SHA1_SLIDING] * len(units)
    plist = [C.params(window_bytes=w, mask=mask, target=target, chunk_segment_bytes=16)] * len(units)
    outs = [C.out_bytes(SHA1_SLIDING, len(u), plist[0]) for u in units]
    got = _run(torch_cuda, C, units, kinds, plist, out_sizes=outs, align=[0, 3, 1, 2])
    want = _oracle_all(oracle_mod, units, kinds, plist, outs)
    _compare(units, kinds, got, want)


def test_md5_and_sha1_mixed_batch(torch_cuda, C, oracle_mod):
    units, kinds, plist, outs = [], [], [], []
    for i in range(32):
        n = [0, 33, 4097, 70001, 1 << 20, 3000][i % 6] + i
        units.append(_rand(9000 + i, n))
        k = [C.CRYSTAL_KIND_MD5_DIRECT, SHA1_DIRECT, C.CRYSTAL_KIND_MD5_SLIDING, SHA1_SLIDING][i % 4]
        kinds.append(k)
        if k in (2, 4):
            plist.append(C.params(window_bytes=[20, 9][i % 2 if k == 2 else 0], mask=0xFF, target=i & 0xFF,
                                  chunk_segment_bytes=[4096, 700][i % 2]))
            outs.append(C.sliding_out_bytes(n, n // 64 + 4, k))
        else:
            plist.append(C.params(segment_bytes=[4096, 999][i % 2]))
            outs.append(C.digest_size(k))
    got = _run(torch_cuda, C, units, kinds, plist, out_sizes=outs, align=[0, 1, 16, 3])
    want = _oracle_all(oracle_mod, units, kinds, plist, outs)
    _compare(units, kinds, got, want)


def test_largest_units_full_oracle(torch_cuda, C, oracle_mod):
    """The largest units the workloads use (64 MiB, the cap of the served
    request sizes; a 64 MiB direct unit; a 16 MiB SHA-1 sliding unit), ragged
    by a few bytes and misaligned, every output byte against the oracle."""
    sizes = [(64 << 20) + 13, (64 << 20) - 5, (16 << 20) + 3]
    kinds = [SLIDING, DIRECT, SHA1_SLIDING]
    units = [_rand(9100 + i, n) for i, n in enumerate(sizes)]
    plist = [C.params()] * 3
    outs = [C.sliding_out_bytes(sizes[0], sizes[0] // 4096 + 64), 16,
            C.sliding_out_bytes(sizes[2], sizes[2] // 4096 + 64, SHA1_SLIDING)]
    got = _run(torch_cuda, C, units, kinds, plist, out_sizes=outs, align=[3, 0, 9])
    want = _oracle_all(oracle_mod, units, kinds, plist, outs)
    assert [st for st, _ in want] == [0, 0, 0]
    _compare(units, kinds, got, want)


def test_golden_cases_on_gpu(torch_cuda, C):
    """Every stored oracle case (tests/golden/oracle_cases.txt) through the
    CUDA path in one batch: same status and the same used output bytes."""
    import hashlib

    from paper_1005_1695_b300 import inputs
    from test_golden import CASES

    units = [inputs.uniform_unit(c["seed"], 0, c["n"]) for c in CASES]
    kinds = [c["kind"] for c in CASES]
    plist = [C.params(segment_bytes=c["seg"], window_bytes=c["window"], mask=c["mask"], target=c["target"],
                      chunk_segment_bytes=c["cseg"]) for c in CASES]
    outs = [c["out_size"] for c in CASES]
    got = _run(torch_cuda, C, units, kinds, plist, out_sizes=outs, align=[0, 3, 8, 13])
    for c, g in zip(CASES, got):
        if c["kind"] in (2, 4):
            assert int.from_bytes(g[4:8], "little") == c["status"], c
        assert hashlib.sha256(g[:c["used"]]).hexdigest() == c["sha"], c


@pytest.mark.parametrize("kind", [SLIDING, SHA1_SLIDING])
def test_many_small_units_more_tiles_than_the_grid(torch_cuda, C, oracle_mod, kind):
    """3,000 sliding units of 1 B - 6 KiB (about 5,000 tiles, several per CTA of the
    window kernel, their owners hundreds of units apart) with windows of 20 and of
    other lengths, at odd input alignments: every unit against the oracle."""
    rng = np.random.default_rng(17)
    sizes = [int(x) for x in rng.integers(1, 6144, 3000)]
    units = [_rand(20000 + i, n) for i, n in enumerate(sizes)]
    kinds = [kind] * len(units)
    plist = [C.params(window_bytes=[20, 20, 20, 7, 33][i % 5], mask=0x3F, target=0x15) for i in range(len(units))]
    outs = [C.sliding_out_bytes(n, n // 16 + 8, kind) for n in sizes]
    got = _run(torch_cuda, C, units, kinds, plist, out_sizes=outs, align=[0, 1, 6, 11, 15])
    want = _oracle_all(oracle_mod, units, kinds, plist, outs)
    _compare(units, kinds, got, want)
