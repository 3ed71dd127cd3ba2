"""Shared test helpers: layout parsing only, no hashing arithmetic."""
import numpy as np


def used_bytes(kind: int, n: int, out: bytes) -> int:
    """Bytes of an output buffer that carry results (the rest is capacity)."""
    digest = 20 if kind in (3, 4) else 16
    if kind in (1, 3):
        return digest
    if kind == 0:
        return 0
    words = (n + 31) // 32
    n_chunks = int.from_bytes(out[0:4], "little")
    flags = int.from_bytes(out[4:8], "little")
    return 8 + 4 * words + (0 if flags & 1 else (4 + digest) * n_chunks)


def same_result(kind: int, n: int, got: bytes, want: bytes) -> bool:
    u = used_bytes(kind, n, want)
    return len(got) >= u and got[:u] == want[:u]


def first_difference(kind: int, n: int, got: bytes, want: bytes) -> str:
    u = used_bytes(kind, n, want)
    g = np.frombuffer(got[:u], dtype=np.uint8)
    w = np.frombuffer(want[:u], dtype=np.uint8)
    if g.size != w.size:
        return f"size {g.size} != {w.size}"
    bad = np.nonzero(g != w)[0]
    if bad.size == 0:
        return "equal"
    i = int(bad[0])
    return f"first differing byte {i} of {u} (got {g[i]:#x}, want {w[i]:#x}); {bad.size} bytes differ"
