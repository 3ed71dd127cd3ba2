"""CPU oracle for the CrystalGPU hashing hot path -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never routes through
it.  It wraps ``oracle.c`` (plain C, built with gcc) through ctypes and adds the
sequential FIFO job loop.

What each function restates:

* :func:`md5` -- MD5 per RFC 1321 (padding, length, four rounds).
* :func:`sha1` -- SHA-1 per FIPS 180-4 (the hash of the paper's experiments,
  Section 5.2); kinds 3 and 4 are the SHA-1 forms of direct and sliding.
* :func:`direct` -- direct hashing: MD5 over the concatenated per-segment MD5
  digests (StoreGPU's direct hashing, used in Section 5.2 of the paper).
* :func:`sliding_bitmap`, :func:`chunk_ends`, :func:`task` -- sliding-window
  hashing with content-defined chunk boundaries (the hashing-based primitives
  for content-addressable storage, Section 2.2).
* :func:`run_tasks` -- the job loop of Section 4.2 (jobs taken from the
  outstanding queue in FIFO order, each one copied in, processed, copied out)
  executed one job at a time on the host.

The readings taken where the paper is silent are listed in ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Iterable, List, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

KIND_NOP = 0
KIND_MD5_DIRECT = 1
KIND_MD5_SLIDING = 2
KIND_SHA1_DIRECT = 3
KIND_SHA1_SLIDING = 4
HASH_MD5 = 0
HASH_SHA1 = 1

_u8p = ctypes.POINTER(ctypes.c_uint8)
_u32p = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` with gcc (plain -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-Wall", "-Wextra", _SRC, "-o", tmp, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_md5.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
        lib.oracle_md5.restype = None
        lib.oracle_md5_table.argtypes = [ctypes.c_void_p]
        lib.oracle_md5_table.restype = None
        lib.oracle_num_segments.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.oracle_num_segments.restype = ctypes.c_uint64
        lib.oracle_direct.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p]
        lib.oracle_direct.restype = ctypes.c_int
        lib.oracle_sliding_bitmap.argtypes = [
            ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
            ctypes.c_void_p,
        ]
        lib.oracle_sliding_bitmap.restype = None
        lib.oracle_chunk_ends.argtypes = [
            ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint64,
        ]
        lib.oracle_chunk_ends.restype = ctypes.c_uint64
        lib.oracle_task.argtypes = [
            ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
            ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint64,
        ]
        lib.oracle_task.restype = ctypes.c_int
        lib.oracle_sha1.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
        lib.oracle_sha1.restype = None
        lib.oracle_direct_hash.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                           ctypes.c_void_p]
        lib.oracle_direct_hash.restype = ctypes.c_int
        lib.oracle_sliding_bitmap_hash.argtypes = [
            ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
            ctypes.c_void_p,
        ]
        lib.oracle_sliding_bitmap_hash.restype = None
        lib.oracle_digest_bytes.argtypes = [ctypes.c_int]
        lib.oracle_digest_bytes.restype = ctypes.c_uint32
        _lib = lib
    return _lib


def _buf(data) -> Tuple[np.ndarray, int]:
    arr = np.frombuffer(memoryview(data), dtype=np.uint8) if not isinstance(data, np.ndarray) else data
    arr = np.ascontiguousarray(arr, dtype=np.uint8)
    return arr, arr.ctypes.data


def md5(data) -> bytes:
    """MD5 digest (16 bytes) of ``data`` (RFC 1321)."""
    arr, p = _buf(data)
    out = (ctypes.c_uint8 * 16)()
    _load().oracle_md5(p, arr.size, out)
    return bytes(out)


def sha1(data) -> bytes:
    """SHA-1 digest (20 bytes) of ``data`` (FIPS 180-4)."""
    arr, p = _buf(data)
    out = (ctypes.c_uint8 * 20)()
    _load().oracle_sha1(p, arr.size, out)
    return bytes(out)


def digest_bytes(kind: int) -> int:
    return 20 if kind in (KIND_SHA1_DIRECT, KIND_SHA1_SLIDING) else 16


def hash_of(kind: int) -> int:
    return HASH_SHA1 if kind in (KIND_SHA1_DIRECT, KIND_SHA1_SLIDING) else HASH_MD5


def md5_table() -> List[int]:
    """The oracle's 64 sine-derived constants, for the closed-form pin."""
    out = (ctypes.c_uint32 * 64)()
    _load().oracle_md5_table(out)
    return list(out)


def num_segments(n: int, seg_bytes: int) -> int:
    return int(_load().oracle_num_segments(n, seg_bytes))


def direct(data, seg_bytes: int = 4096, hash: int = HASH_MD5) -> bytes:
    """Direct hash: H over the concatenated H digests of ``seg_bytes``
    segments (H = MD5 or SHA-1)."""
    arr, p = _buf(data)
    out = (ctypes.c_uint8 * 20)()
    if _load().oracle_direct_hash(hash, p, arr.size, seg_bytes, out) != 0:
        raise ValueError("oracle_direct failed")
    return bytes(out)[:20 if hash == HASH_SHA1 else 16]


def sliding_bitmap(data, window: int = 20, mask: int = 0x1FFF, target: int = 0x1FFF,
                   hash: int = HASH_MD5) -> np.ndarray:
    """Boundary bitmap, ``ceil(n/32)`` little-endian uint32 words."""
    arr, p = _buf(data)
    words = (arr.size + 31) // 32
    bm = np.zeros(max(words, 1), dtype=np.uint32)
    _load().oracle_sliding_bitmap_hash(hash, p, arr.size, window, mask, target, bm.ctypes.data)
    return bm[:words]


def chunk_ends(bitmap: np.ndarray, n: int, window: int) -> np.ndarray:
    """Sorted chunk ends ``{i + w : bit i} U {n}`` (duplicates removed)."""
    bm = np.ascontiguousarray(bitmap, dtype=np.uint32)
    if bm.size == 0:
        bm = np.zeros(1, dtype=np.uint32)
    lib = _load()
    count = int(lib.oracle_chunk_ends(bm.ctypes.data, n, window, None, 0))
    ends = np.zeros(count, dtype=np.uint32)
    lib.oracle_chunk_ends(bm.ctypes.data, n, window, ends.ctypes.data, count)
    return ends


def sliding_out_bytes(n: int, max_chunks: int, digest: int = 16) -> int:
    """Output-buffer bytes for a sliding job that can hold ``max_chunks`` records
    (``digest`` = 16 for MD5, 20 for SHA-1)."""
    return 8 + 4 * ((n + 31) // 32) + (4 + digest) * max_chunks


def task(kind: int, data, out_size: int, seg_bytes: int = 4096, window: int = 20,
         mask: int = 0x1FFF, target: int = 0x1FFF, chunk_seg_bytes: int = 4096) -> Tuple[int, bytes]:
    """One job, synchronously: returns ``(status, out_bytes)``.

    status 0 = OK, 1 = chunk records did not fit (header still holds the
    needed count), -1 = bad argument."""
    arr, p = _buf(data)
    out = np.zeros(max(out_size, 1), dtype=np.uint8)
    st = _load().oracle_task(kind, p, arr.size, seg_bytes, window, mask, target, chunk_seg_bytes,
                             out.ctypes.data, out_size)
    return int(st), out[:out_size].tobytes()


def parse_sliding(out: bytes, n: int, digest: int = 16):
    """Split a sliding output buffer into (n_chunks, flags, bitmap, ends, digests)."""
    hdr = np.frombuffer(out[:8], dtype=np.uint32)
    n_chunks, flags = int(hdr[0]), int(hdr[1])
    words = (n + 31) // 32
    bm = np.frombuffer(out[8:8 + 4 * words], dtype=np.uint32)
    if flags & 1:
        return n_chunks, flags, bm, None, None
    off = 8 + 4 * words
    ends = np.frombuffer(out[off:off + 4 * n_chunks], dtype=np.uint32)
    off += 4 * n_chunks
    dig = np.frombuffer(out[off:off + digest * n_chunks], dtype=np.uint8).reshape(n_chunks, digest)
    return n_chunks, flags, bm, ends, dig


def run_tasks(jobs: Iterable[Tuple[int, object, int, dict]]) -> List[Tuple[int, bytes]]:
    """The job loop, one job at a time in FIFO order.

    ``jobs`` yields ``(kind, data, out_size, params)``; the result list keeps
    submission order.  A job's result depends only on its own bytes, kind
    and parameters."""
    results = []
    for kind, data, out_size, params in jobs:
        results.append(task(kind, data, out_size, **params))
    return results


def run_tasks_parallel(jobs: Sequence[Tuple[int, object, int, dict]], threads: int) -> List[Tuple[int, bytes]]:
    """Same results as :func:`run_tasks`, jobs spread over host threads
    (ctypes releases the GIL inside each C call)."""
    from concurrent.futures import ThreadPoolExecutor

    if threads <= 1:
        return run_tasks(jobs)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(lambda j: task(j[0], j[1], j[2], **j[3]), jobs))
