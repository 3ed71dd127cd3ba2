"""The C-ABI library on a machine without a GPU: it loads, exports every
function ``include/crystal.h`` declares, and its host-only logic (arena
allocator, batch planning, size arithmetic, status strings) behaves.  No
call here touches a CUDA device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "crystal.h")


@pytest.fixture(scope="module")
def C():
    from paper_1005_1695_b300 import crystal

    crystal.load()
    return crystal


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(crystal_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_paper_api():
    names = declared_functions()
    for n in ["crystal_init", "crystal_shutdown", "crystal_task_create", "crystal_task_submit",
              "crystal_task_poll", "crystal_task_wait", "crystal_task_release", "crystal_task_host_in",
              "crystal_task_host_out", "crystal_out_bytes", "crystal_strerror"]:
        assert n in names


def test_library_exports_every_declared_symbol(C):
    lib = ctypes.CDLL(C.lib_path())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_sizes_match_header(C):
    assert ctypes.sizeof(C.crystal_config) == 64
    assert ctypes.sizeof(C.crystal_hash_params) == 24
    assert C.UNIT_DTYPE.itemsize == 64
    assert C.load().crystal_batch_bytes(3) == 64 + 3 * 64


def test_strerror_covers_codes(C):
    L = C.load()
    for code in range(-7, 2):
        assert L.crystal_strerror(code)
    assert L.crystal_strerror(-99) == b"unknown status"


def _arena(C, size, align=256):
    L = C.load()
    h = ctypes.c_void_p()
    assert L.crystal_arena_create(size, align, ctypes.byref(h)) == 0
    return L, h


def _alloc(L, h, n):
    off = ctypes.c_uint64()
    st = L.crystal_arena_alloc(h, n, ctypes.byref(off))
    return st, off.value


def test_arena_alloc_free_coalesce(C):
    L, h = _arena(C, 1 << 20)
    offs = []
    for _ in range(16):
        st, o = _alloc(L, h, 65536)
        assert st == 0
        offs.append(o)
    assert sorted(offs) == [i * 65536 for i in range(16)]
    assert _alloc(L, h, 1)[0] == C.CRYSTAL_EAGAIN
    assert L.crystal_arena_used(h) == 1 << 20
    for o in offs[::2]:
        assert L.crystal_arena_free(h, o) == 0
    assert L.crystal_arena_largest_free(h) == 65536
    assert _alloc(L, h, 65537)[0] == C.CRYSTAL_EAGAIN
    for o in offs[1::2]:
        assert L.crystal_arena_free(h, o) == 0
    assert L.crystal_arena_used(h) == 0
    assert L.crystal_arena_largest_free(h) == 1 << 20
    assert L.crystal_arena_free(h, 12345) == C.CRYSTAL_EINVAL
    L.crystal_arena_destroy(h)


def test_arena_alignment_and_random_churn(C):
    L, h = _arena(C, 64 << 20, 256)
    rng = np.random.default_rng(0)
    live = {}
    for step in range(4000):
        if live and (rng.random() < 0.45 or len(live) > 200):
            o = int(rng.choice(list(live)))
            assert L.crystal_arena_free(h, o) == 0
            del live[o]
        else:
            n = int(rng.integers(1, 1 << 18))
            st, o = _alloc(L, h, n)
            if st == 0:
                assert o % 256 == 0
                for lo, ln in live.items():
                    assert o + n <= lo or lo + ln <= o, "overlap"
                live[o] = n
    for o in list(live):
        assert L.crystal_arena_free(h, o) == 0
    assert L.crystal_arena_used(h) == 0 and L.crystal_arena_largest_free(h) == 64 << 20
    L.crystal_arena_destroy(h)


def _alloc_at(L, h, n, placement):
    off = ctypes.c_uint64()
    st = L.crystal_arena_alloc_at(h, n, placement, ctypes.byref(off))
    return st, off.value


def test_arena_placement_matches_a_model(C):
    """Random churn with all three placements against a plain model of the
    free list: best fit takes the smallest block that fits (lowest offset on a
    tie) from its bottom, LOWEST the lowest-addressed block that fits from its
    bottom, HIGHEST the highest-addressed one from its top; freed blocks merge
    with free neighbours."""
    L, h = _arena(C, 32 << 20, 256)
    free = {0: 32 << 20}  # offset -> length
    live = {}
    rng = np.random.default_rng(5)

    def model_alloc(want, placement):
        fits = [(o, n) for o, n in free.items() if n >= want]
        if not fits:
            return None
        if placement == 0:
            o, n = min(fits, key=lambda x: (x[1], x[0]))
        elif placement == 1:
            o, n = min(fits)
        else:
            o, n = max(fits)
        del free[o]
        at = o + n - want if placement == 2 else o
        rest = (o, n - want) if placement == 2 else (o + want, n - want)
        if rest[1]:
            free[rest[0]] = rest[1]
        return at

    def model_free(o):
        n = live.pop(o)
        nxt = o + n
        if nxt in free:
            n += free.pop(nxt)
        prev = [p for p, m in free.items() if p + m == o]
        if prev:
            o, n = prev[0], n + free.pop(prev[0])
        free[o] = n

    for step in range(3000):
        if live and (rng.random() < 0.45 or len(live) > 150):
            o = int(rng.choice(sorted(live)))
            assert L.crystal_arena_free(h, o) == 0
            model_free(o)
        else:
            n = int(rng.integers(1, 1 << 19)) if rng.random() < 0.9 else int(rng.integers(1, 600))
            placement = int(rng.integers(0, 4))
            want = (n + 255) // 256 * 256
            if placement == 3:  # exactly at an offset: inside one free block, or refused
                at = int(rng.integers(0, (32 << 20) // 256)) * 256
                holder = [(fo, fn) for fo, fn in free.items() if fo <= at and at + want <= fo + fn]
                st = L.crystal_arena_alloc_exact(h, at, n)
                if not holder:
                    assert st == C.CRYSTAL_EAGAIN
                    continue
                assert st == 0
                fo, fn = holder[0]
                del free[fo]
                if at > fo:
                    free[fo] = at - fo
                if fo + fn > at + want:
                    free[at + want] = fo + fn - at - want
                live[at] = want
                continue
            expect = model_alloc(want, placement)
            st, o = _alloc_at(L, h, n, placement)
            if expect is None:
                assert st == C.CRYSTAL_EAGAIN
            else:
                assert st == 0 and o == expect, (step, placement, n, o, expect)
                live[o] = want
        assert L.crystal_arena_largest_free(h) == max(free.values(), default=0)
    assert L.crystal_arena_alloc_exact(h, 100, 10) == C.CRYSTAL_EINVAL  # off the 256-byte alignment
    assert L.crystal_arena_alloc_exact(h, 32 << 20, 1) == C.CRYSTAL_EAGAIN  # past the end
    L.crystal_arena_destroy(h)


def test_sizes(C):
    p = C.params()
    assert C.out_bytes(C.CRYSTAL_KIND_MD5_DIRECT, 12345, p) == 16
    n = 1 << 20
    assert C.sliding_out_bytes(n, 0) == 8 + 4 * (n // 32)
    assert C.out_bytes(C.CRYSTAL_KIND_MD5_SLIDING, n, p) == 8 + 4 * (n // 32) + 20 * (n - 20 + 2)
    assert C.out_bytes(C.CRYSTAL_KIND_MD5_SLIDING, 5, p) == 8 + 4 + 20
    assert C.scratch_bytes(C.CRYSTAL_KIND_MD5_DIRECT, 65536, 16, p) == 16 * 16
    assert C.scratch_bytes(C.CRYSTAL_KIND_MD5_DIRECT, 0, 16, p) == 16
    out = C.sliding_out_bytes(n, 1000)
    cap = 1000
    assert C.scratch_bytes(C.CRYSTAL_KIND_MD5_SLIDING, n, out, p) == \
        ((4 * (cap + 1) + 15) // 16 * 16) + 16 * (cap + n // 4096 + 1)


def _plan(C, units, nd, ns):
    buf = np.zeros(64 + 64 * len(units), dtype=np.uint8)
    rec = buf[64:].view(C.UNIT_DTYPE)
    for i, u in enumerate(units):
        for k, v in u.items():
            rec[i][k] = v
    st = C.load().crystal_batch_plan(buf.ctypes.data, nd, ns)
    return st, buf, rec


def _unit(kind, n, **kw):
    u = {"in": 1 << 20, "n": n, "out": 2 << 20, "scratch": 3 << 20, "out_cap": 1 << 20,
         "seg_bytes": 4096, "window": 20, "mask": 0x1FFF, "target": 0x1FFF, "kind": kind}
    u.update(kw)
    return u


def test_batch_plan_prefixes_and_validation(C):
    D, S = C.CRYSTAL_KIND_MD5_DIRECT, C.CRYSTAL_KIND_MD5_SLIDING
    units = [_unit(D, 0), _unit(D, 4096), _unit(D, 4097), _unit(D, 100, seg_bytes=7),
             _unit(S, 0), _unit(S, 1024), _unit(S, 1025), _unit(S, 10, window=55)]
    tile = int(re.search(r"#define CRYSTAL_SLIDING_TILE (\d+)u", open(HEADER).read()).group(1))
    st, buf, rec = _plan(C, units, 4, 4)
    assert st == 0
    sl_tiles = [-(-n // tile) for n in (0, 1024, 1025, 10)]
    sl_begin = [int(v) for v in np.cumsum([0] + sl_tiles[:-1])]
    assert rec["work_begin"].tolist() == [0, 1, 2, 4] + sl_begin
    hdr = buf[:64]
    assert hdr[:8].view("<u4").tolist() == [4, 4]
    assert hdr[8:24].view("<u8").tolist() == [4 + 15, sum(sl_tiles)]
    assert hdr[24:28].view("<u4")[0] == 55
    assert hdr[32:40].view("<u8")[0] == sum(sl_tiles[:3])  # tiles of the w = 20 units


def test_batch_plan_puts_w20_units_first(C):
    D, S = C.CRYSTAL_KIND_MD5_DIRECT, C.CRYSTAL_KIND_MD5_SLIDING
    units = [_unit(S, 5000, window=7, out=1 << 21), _unit(S, 3000, out=2 << 21), _unit(S, 100, window=33, out=3 << 21),
             _unit(S, 9000, out=4 << 21)]
    st, buf, rec = _plan(C, units, 0, 4)
    assert st == 0
    assert rec["window"].tolist() == [20, 20, 7, 33]
    assert rec["out"].tolist() == [2 << 21, 4 << 21, 1 << 21, 3 << 21]  # records move whole
    bad = [
        [_unit(S, 10)] + units[1:4],               # wrong kind order
        [_unit(D, 10, seg_bytes=0)],               # zero segment
        [_unit(D, 10, scratch=(3 << 20) + 8)],     # misaligned scratch
        [_unit(D, 10, out_cap=15)],                # direct output < 16
    ]
    for b in bad:
        assert _plan(C, b, len(b), 0)[0] == C.CRYSTAL_EINVAL
    for b in ([_unit(S, 10, window=56)], [_unit(S, 10, window=0)], [_unit(S, 4096, out_cap=100)],
              [_unit(S, 1 << 32)]):
        assert _plan(C, b, 0, 1)[0] == C.CRYSTAL_EINVAL


def test_batch_plan_orders_hashes(C):
    D5, S5, D1, S1 = (C.CRYSTAL_KIND_MD5_DIRECT, C.CRYSTAL_KIND_MD5_SLIDING, C.CRYSTAL_KIND_SHA1_DIRECT,
                      C.CRYSTAL_KIND_SHA1_SLIDING)
    units = [_unit(D1, 5000, out=1 << 21), _unit(D5, 4096, out=2 << 21), _unit(D1, 100, out=3 << 21),
             _unit(S1, 3000, out=4 << 21), _unit(S5, 9000, window=7, out=5 << 21), _unit(S5, 5000, out=6 << 21)]
    st, buf, rec = _plan(C, units, 3, 3)
    assert st == 0
    assert rec["kind"].tolist() == [D5, D1, D1, S5, S5, S1]
    assert rec["window"].tolist()[3:] == [20, 7, 20]
    hdr = buf[:64]
    tile = int(re.search(r"#define CRYSTAL_SLIDING_TILE (\d+)u", open(HEADER).read()).group(1))
    t = [-(-n // tile) for n in (5000, 9000, 3000)]
    assert hdr[32:40].view("<u8")[0] == t[0]                 # MD5 w = 20 tiles
    assert hdr[48:56].view("<u8")[0] == t[0] + t[1]          # all MD5 sliding tiles
    assert hdr[56:64].view("<u8")[0] == 1                    # MD5 direct segments (one 4096-byte unit)
    assert hdr[8:16].view("<u8")[0] == 1 + 2 + 1             # all direct segments
    bad = [_unit(D1, 10, out_cap=19)]                        # SHA-1 digest needs 20 bytes
    assert _plan(C, bad, 1, 0)[0] == C.CRYSTAL_EINVAL


def test_sha1_sizes(C):
    n = 1 << 20
    assert C.out_bytes(C.CRYSTAL_KIND_SHA1_DIRECT, n) == 20
    assert C.sliding_out_bytes(n, 10, C.CRYSTAL_KIND_SHA1_SLIDING) == 8 + 4 * (n // 32) + 24 * 10
    assert C.scratch_bytes(C.CRYSTAL_KIND_SHA1_DIRECT, 65536, 20) == 20 * 16


def test_arena_two_ended_placement(C):
    L, h = _arena(C, 1 << 20)
    off = ctypes.c_uint64()
    lows, highs = [], []
    for i in range(6):
        assert L.crystal_arena_alloc_at(h, 1000, 1, ctypes.byref(off)) == 0
        lows.append(off.value)
        assert L.crystal_arena_alloc_at(h, 3000, 2, ctypes.byref(off)) == 0
        highs.append(off.value)
    assert lows == [1024 * i for i in range(6)]                        # ascending, adjacent
    assert highs == [(1 << 20) - 3072 * (i + 1) for i in range(6)]      # descending, adjacent
    assert L.crystal_arena_alloc_at(h, 10, 3, ctypes.byref(off)) == C.CRYSTAL_EINVAL
    for o in lows + highs:
        assert L.crystal_arena_free(h, o) == 0
    assert L.crystal_arena_largest_free(h) == 1 << 20
    assert L.crystal_arena_alloc_at(h, 2 << 20, 2, ctypes.byref(off)) == C.CRYSTAL_EAGAIN
    L.crystal_arena_destroy(h)


def test_arena_top_blocks_aligned_for_any_size(C):
    L, h = _arena(C, (1 << 20) + 1000)  # not a multiple of the alignment
    off = ctypes.c_uint64()
    for _ in range(5):
        assert L.crystal_arena_alloc_at(h, 777, 2, ctypes.byref(off)) == 0
        assert off.value % 256 == 0
    L.crystal_arena_destroy(h)


def test_entry_points_refuse_missing_arguments_on_the_host(C):
    """Every entry point that takes a context, job or batch refuses a NULL one
    (and the other missing arguments each documents) with CRYSTAL_EINVAL
    before any device call, so these run without a GPU."""
    L = C.load()
    EINVAL = C.CRYSTAL_EINVAL
    h = ctypes.c_void_p()
    assert L.crystal_init(None, ctypes.byref(h)) == EINVAL
    cfg = C.crystal_config()
    L.crystal_config_default(ctypes.byref(cfg))
    assert L.crystal_init(ctypes.byref(cfg), None) == EINVAL
    assert L.crystal_shutdown(None) == EINVAL
    for name in ("crystal_task_poll", "crystal_task_release", "crystal_prepare_graphs"):
        assert getattr(L, name)(None) == EINVAL, name
    assert L.crystal_task_wait(None, 0) == EINVAL
    assert L.crystal_task_wait_many(None, 1, 0) == EINVAL
    assert L.crystal_task_wait_many(None, 0, 0) == C.CRYSTAL_OK  # nothing to wait for
    assert L.crystal_task_resize(None, 0, 0) == EINVAL
    assert L.crystal_task_bind_input(None, None, 0) == EINVAL
    assert L.crystal_task_timing(None, None, None, None) == EINVAL
    assert L.crystal_task_set_priority(None, 1) == EINVAL
    assert L.crystal_task_submit(None, C.CRYSTAL_KIND_MD5_DIRECT, None, C.crystal_callback(), None) == EINVAL
    assert L.crystal_get_stats(None, None) == EINVAL
    assert L.crystal_get_config(None, None) == EINVAL
    assert L.crystal_set_geometry(None, 0, None) == EINVAL
    res = np.zeros(1, dtype=C.RESULT_DTYPE)
    assert L.crystal_serve(None, None, 0, None, 0, None, res.ctypes.data, None) == EINVAL
    assert L.crystal_stream_staged(None, None, None, 0, None, None, 0, res.ctypes.data, None) == EINVAL
    for name in ("crystal_launch_direct", "crystal_launch_direct_segments", "crystal_launch_direct_outer",
                 "crystal_launch_sliding", "crystal_launch_sliding_windows", "crystal_launch_sliding_chunks",
                 "crystal_launch_sliding_digests", "crystal_launch_batch"):
        assert getattr(L, name)(None, None) == EINVAL, name
    assert L.crystal_alu_probe(0, 2, 1, 0, None, None, None) == EINVAL   # no sink
    assert L.crystal_alu_probe(0, 0, 1, 0, 16, None, None) == EINVAL     # no CTAs
    assert L.crystal_alu_probe(0, 2, 0, 0, 16, None, None) == EINVAL     # no iterations
    assert L.crystal_md5_direct_noalloc(None, 4096, 1, 4096, None, None) == EINVAL
    assert L.crystal_md5_direct_noalloc(None, 4096, 0, 4096, None, None) == C.CRYSTAL_OK  # no units
