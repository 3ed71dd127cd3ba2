"""Pins for the CPU oracle against things other than itself.

* MD5: the sine-derived constants against their closed form evaluated in
  50-digit arithmetic; digests against Python's ``hashlib`` (an independent
  MD5 implementation that is run, never read) over every padding branch.
* Direct hashing: the closed form written with ``hashlib`` and the special
  sizes n = 0, n < S, n = S, n = S + 1, n = k*S.
* Sliding window: brute-force enumeration of every window with ``hashlib``
  on tiny inputs (every n <= 64, w in {1, 2, 3, 20}, several masks), cut sets
  from a plain set construction, and invariants that hold at any size
  (chunks tile the unit, popcount = cuts, boundary spacing ~ 2^13 on random
  data, repeated content gives repeated chunk digests).
"""
import hashlib
import struct

import numpy as np
import pytest

from paper_1005_1695_b300 import inputs


def _bytes(seed, n):
    return inputs.uniform_unit(seed, 7, n).tobytes()


# ---- MD5 ------------------------------------------------------------------

def test_md5_constant_table_closed_form(oracle_mod):
    import mpmath

    mpmath.mp.dps = 50
    want = [int(mpmath.floor(abs(mpmath.sin(i + 1)) * 2 ** 32)) for i in range(64)]
    assert oracle_mod.md5_table() == want


@pytest.mark.parametrize("n", list(range(0, 201)))
def test_md5_every_length_to_200(oracle_mod, n):
    x = _bytes(n, n)
    assert oracle_mod.md5(x) == hashlib.md5(x).digest()


@pytest.mark.parametrize("fill", [0x00, 0xFF, 0x80])
@pytest.mark.parametrize("n", [1, 55, 56, 57, 63, 64, 65, 119, 120, 121, 127, 128, 4095, 4096, 4097])
def test_md5_constant_bytes(oracle_mod, fill, n):
    x = bytes([fill]) * n
    assert oracle_mod.md5(x) == hashlib.md5(x).digest()


@pytest.mark.parametrize("seed", range(6))
def test_md5_random_lengths(oracle_mod, seed):
    g = np.random.default_rng(seed)
    n = int(g.integers(1, 1 << 20))
    x = _bytes(seed + 100, n)
    assert oracle_mod.md5(x) == hashlib.md5(x).digest()


# ---- direct hashing ---------------------------------------------------------

def direct_closed_form(x: bytes, S: int) -> bytes:
    m = max(1, -(-len(x) // S))
    segs = [x[i * S:(i + 1) * S] for i in range(m)]
    return hashlib.md5(b"".join(hashlib.md5(s).digest() for s in segs)).digest()


@pytest.mark.parametrize("S", [64, 100, 4096])
def test_direct_special_sizes(oracle_mod, S):
    for n in [0, 1, S - 1, S, S + 1, 2 * S, 3 * S - 7, 16 * S]:
        x = _bytes(n + S, n)
        assert oracle_mod.direct(x, S) == direct_closed_form(x, S), (n, S)


def test_direct_empty_is_md5_of_md5_of_empty(oracle_mod):
    assert oracle_mod.direct(b"", 4096) == hashlib.md5(hashlib.md5(b"").digest()).digest()


def test_direct_config_shape(oracle_mod):
    # 64 KiB unit, 4 KiB segments -> 16 inner digests, a 256-byte outer message
    x = _bytes(1, 65536)
    assert oracle_mod.num_segments(65536, 4096) == 16
    assert oracle_mod.direct(x, 4096) == direct_closed_form(x, 4096)
    assert oracle_mod.direct(x, 4096) != hashlib.md5(x).digest()


# ---- sliding window -------------------------------------------------------

def brute_bitmap(x: bytes, w: int, mask: int, target: int):
    n = len(x)
    bits = []
    for i in range(0, n - w + 1) if n >= w else []:
        word0 = struct.unpack("<I", hashlib.md5(x[i:i + w]).digest()[:4])[0]
        if (word0 & mask) == target:
            bits.append(i)
    return bits


def words_from_bits(bits, n):
    words = np.zeros((n + 31) // 32, dtype=np.uint32)
    for i in bits:
        words[i // 32] |= np.uint32(1 << (i % 32))
    return words


def brute_ends(bits, n, w):
    return sorted({i + w for i in bits} | {n})


@pytest.mark.parametrize("w", [1, 2, 3, 20])
@pytest.mark.parametrize("mask,target", [(0x0, 0x0), (0x1, 0x1), (0x3, 0x0), (0x3, 0x3), (0x1FFF, 0x1FFF)])
def test_sliding_bruteforce_tiny(oracle_mod, w, mask, target):
    for n in range(0, 65):
        x = _bytes(1000 + n, n)
        bits = brute_bitmap(x, w, mask, target)
        bm = oracle_mod.sliding_bitmap(x, w, mask, target)
        assert np.array_equal(bm, words_from_bits(bits, n)), (n, w, mask)
        ends = oracle_mod.chunk_ends(bm, n, w)
        assert list(ends) == brute_ends(bits, n, w), (n, w, mask)


def test_sliding_mask_zero_marks_every_window(oracle_mod):
    x = _bytes(5, 100)
    bm = oracle_mod.sliding_bitmap(x, 20, 0, 0)
    bits = [i for i in range(100) if bm[i // 32] >> (i % 32) & 1]
    assert bits == list(range(0, 81))
    ends = oracle_mod.chunk_ends(bm, 100, 20)
    assert list(ends) == list(range(20, 101))


def test_sliding_unit_shorter_than_window(oracle_mod):
    for n in range(0, 20):
        x = _bytes(n, n)
        bm = oracle_mod.sliding_bitmap(x, 20, 0, 0)
        assert not bm.any()
        assert list(oracle_mod.chunk_ends(bm, n, 20)) == [n]


def _parse(oracle_mod, out, n):
    return oracle_mod.parse_sliding(out, n)


@pytest.mark.parametrize("seed", [1, 2])
def test_sliding_task_layout_and_chunk_digests(oracle_mod, seed):
    n = 5000
    x = _bytes(seed, n)
    w, mask, target, S = 20, 0x3F, 0x3F, 100
    bits = brute_bitmap(x, w, mask, target)
    ends = brute_ends(bits, n, w)
    out_size = oracle_mod.sliding_out_bytes(n, len(ends) + 3)
    st, out = oracle_mod.task(oracle_mod.KIND_MD5_SLIDING, x, out_size, window=w, mask=mask,
                              target=target, chunk_seg_bytes=S)
    assert st == 0
    n_chunks, flags, bm, e, dig = _parse(oracle_mod, out, n)
    assert flags == 0 and n_chunks == len(ends)
    assert np.array_equal(bm, words_from_bits(bits, n))
    assert list(e) == ends
    start = 0
    for k, end in enumerate(ends):
        assert dig[k].tobytes() == direct_closed_form(x[start:end], S)
        start = end


def test_sliding_task_overflow_keeps_count(oracle_mod):
    n = 3000
    x = _bytes(9, n)
    bits = brute_bitmap(x, 20, 0x7, 0x7)
    need = len(brute_ends(bits, n, 20))
    out_size = oracle_mod.sliding_out_bytes(n, need - 1)
    st, out = oracle_mod.task(oracle_mod.KIND_MD5_SLIDING, x, out_size, window=20, mask=0x7, target=0x7)
    assert st == 1
    n_chunks, flags, bm, _, _ = _parse(oracle_mod, out, n)
    assert flags == 1 and n_chunks == need
    assert np.array_equal(bm, words_from_bits(bits, n))
    st2, _ = oracle_mod.task(oracle_mod.KIND_MD5_SLIDING, x, out_size + 20, window=20, mask=0x7, target=0x7)
    assert st2 == 0


def test_sliding_invariants_random_mib(oracle_mod):
    """4 MiB of random bytes: chunks tile [0, n), popcount(bitmap) = cuts, and
    the number of boundaries is Binomial(n - w + 1, 2^-13) within 6 sigma."""
    n = 4 << 20
    x = inputs.uniform_unit(3, 0, n)
    bm = oracle_mod.sliding_bitmap(x, 20, 0x1FFF, 0x1FFF)
    ends = oracle_mod.chunk_ends(bm, n, 20)
    pop = int(sum(bin(int(v)).count("1") for v in bm))
    assert ends[-1] == n and np.all(np.diff(ends.astype(np.int64)) > 0)
    assert len(ends) == pop + (0 if (bm[(n - 20) // 32] >> ((n - 20) % 32)) & 1 else 1)
    p = 2.0 ** -13
    windows = n - 20 + 1
    mean, sd = windows * p, (windows * p * (1 - p)) ** 0.5
    assert abs(pop - mean) < 6 * sd, (pop, mean, sd)


def test_sliding_repeated_content_repeats_chunk_digests(oracle_mod):
    """Copies of the same block give the same chunk digests for every chunk
    whose cuts both come from windows inside the copies."""
    w, mask = 20, 0x3F
    block = _bytes(11, 16384)
    x = _bytes(12, 5000) + block + _bytes(13, 7777) + block
    n = len(x)
    starts = [5000, 5000 + 16384 + 7777]
    out_size = oracle_mod.sliding_out_bytes(n, n)
    st, out = oracle_mod.task(oracle_mod.KIND_MD5_SLIDING, x, out_size, window=w, mask=mask, target=mask)
    assert st == 0
    _, _, _, ends, dig = _parse(oracle_mod, out, n)
    per_copy = []
    for s in starts:
        inner = {}
        prev = 0
        for k, e in enumerate(ends):
            e = int(e)
            # both cuts produced by windows fully inside this copy
            if prev - w >= s and e <= s + len(block) and e != n:
                inner[(prev - s, e - s)] = dig[k].tobytes()
            prev = e
        per_copy.append(inner)
    assert len(per_copy[0]) > 50
    assert per_copy[0] == per_copy[1]


def test_run_tasks_fifo_and_pure(oracle_mod):
    jobs = []
    for i in range(6):
        n = 1000 + 37 * i
        kind = oracle_mod.KIND_MD5_DIRECT if i % 2 == 0 else oracle_mod.KIND_MD5_SLIDING
        out = 16 if kind == oracle_mod.KIND_MD5_DIRECT else oracle_mod.sliding_out_bytes(n, n)
        jobs.append((kind, _bytes(i, n), out, dict(seg_bytes=256, mask=0xF, target=0xF)))
    res = oracle_mod.run_tasks(jobs)
    res_rev = oracle_mod.run_tasks(list(reversed(jobs)))
    assert res == list(reversed(res_rev))
    assert res[0][1] == direct_closed_form(jobs[0][1], 256)
    assert oracle_mod.run_tasks_parallel(jobs, 3) == res


# ---- SHA-1 (the hash of the paper's own experiments) ------------------------

@pytest.mark.parametrize("n", list(range(0, 201)))
def test_sha1_every_length_to_200(oracle_mod, n):
    x = _bytes(n + 5000, n)
    assert oracle_mod.sha1(x) == hashlib.sha1(x).digest()


@pytest.mark.parametrize("fill", [0x00, 0xFF])
@pytest.mark.parametrize("n", [55, 56, 63, 64, 119, 120, 4096])
def test_sha1_constant_bytes(oracle_mod, fill, n):
    x = bytes([fill]) * n
    assert oracle_mod.sha1(x) == hashlib.sha1(x).digest()


def test_sha1_random_lengths(oracle_mod):
    g = np.random.default_rng(77)
    for k in range(4):
        x = _bytes(600 + k, int(g.integers(1, 1 << 20)))
        assert oracle_mod.sha1(x) == hashlib.sha1(x).digest()


def sha1_direct_closed_form(x: bytes, S: int) -> bytes:
    m = max(1, -(-len(x) // S))
    return hashlib.sha1(b"".join(hashlib.sha1(x[i * S:(i + 1) * S]).digest() for i in range(m))).digest()


@pytest.mark.parametrize("S", [64, 100, 4096])
def test_sha1_direct_special_sizes(oracle_mod, S):
    for n in [0, 1, S - 1, S, S + 1, 3 * S - 7, 16 * S]:
        x = _bytes(n + 7 * S, n)
        assert oracle_mod.direct(x, S, hash=oracle_mod.HASH_SHA1) == sha1_direct_closed_form(x, S), (n, S)


@pytest.mark.parametrize("w", [1, 3, 20])
@pytest.mark.parametrize("mask,target", [(0x0, 0x0), (0x3, 0x1), (0x1FFF, 0x1FFF)])
def test_sha1_sliding_bruteforce_tiny(oracle_mod, w, mask, target):
    for n in range(0, 49):
        x = _bytes(3000 + n, n)
        bits = [i for i in range(0, n - w + 1)
                if (struct.unpack("<I", hashlib.sha1(x[i:i + w]).digest()[:4])[0] & mask) == target]
        bm = oracle_mod.sliding_bitmap(x, w, mask, target, hash=oracle_mod.HASH_SHA1)
        assert np.array_equal(bm, words_from_bits(bits, n)), (n, w, mask)


def test_sha1_sliding_task_layout(oracle_mod):
    n, w, mask, S = 4000, 20, 0x3F, 100
    x = _bytes(21, n)
    bits = [i for i in range(0, n - w + 1)
            if (struct.unpack("<I", hashlib.sha1(x[i:i + w]).digest()[:4])[0] & mask) == mask]
    ends = brute_ends(bits, n, w)
    out_size = oracle_mod.sliding_out_bytes(n, len(ends), digest=20)
    st, out = oracle_mod.task(oracle_mod.KIND_SHA1_SLIDING, x, out_size, window=w, mask=mask, target=mask,
                              chunk_seg_bytes=S)
    assert st == 0
    cnt, flags, bm, e, dig = oracle_mod.parse_sliding(out, n, digest=20)
    assert cnt == len(ends) and list(e) == ends and flags == 0
    start = 0
    for k, end in enumerate(ends):
        assert dig[k].tobytes() == sha1_direct_closed_form(x[start:end], S)
        start = end
    st, out = oracle_mod.task(oracle_mod.KIND_SHA1_DIRECT, x, 20, seg_bytes=256)
    assert st == 0 and out == sha1_direct_closed_form(x, 256)
    # one record short: 24-byte records (4-byte end + 20-byte digest) must not fit
    st, out = oracle_mod.task(oracle_mod.KIND_SHA1_SLIDING, x, oracle_mod.sliding_out_bytes(n, len(ends) - 1, 20),
                              window=w, mask=mask, target=mask, chunk_seg_bytes=S)
    assert st == 1 and oracle_mod.parse_sliding(out, n, digest=20)[:2] == (len(ends), 1)
