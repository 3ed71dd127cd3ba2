"""Writes ``oracle_cases.txt``: the CPU oracle's outputs on seeded inputs.

The paper prints no worked example (it measures throughput, not digests), so
the stored values here come from the oracle, by this script only: it calls
nothing but ``oracle/`` and the seeded input generator.  Rerun it only when the
oracle's arithmetic changes for a reason RFC 1321, FIPS 180-4 or the paper's
definitions give, and say which in the commit.

Each line: kind seed n seg_bytes window mask target chunk_seg_bytes out_size
status used_bytes sha256(used output bytes) summary, where the summary is the
digest in hex for direct jobs and the chunk count for sliding jobs.  Inputs are
``inputs.uniform_unit(seed, 0, n)``.

    python tests/golden/make_golden.py
"""
import hashlib
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1005_1695_b300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "oracle_cases.txt")

MD5_DIRECT, MD5_SLIDING, SHA1_DIRECT, SHA1_SLIDING = 1, 2, 3, 4


def cases():
    """(kind, seed, n, seg_bytes, window, mask, target, chunk_seg_bytes, max_chunks)."""
    out = []
    seed = 500
    for kind in (MD5_DIRECT, SHA1_DIRECT):
        for S in (64, 4096):
            for n in (0, 1, 55, 56, 63, 64, 65, 119, 120, 4095, 4096, 4097, 65543):
                seed += 1
                out.append((kind, seed, n, S, 20, 0, 0, 4096, 0))
    for kind in (MD5_SLIDING, SHA1_SLIDING):
        for w, mask, target in ((1, 0x3, 0x1), (20, 0x0, 0x0), (20, 0x3F, 0x3F), (20, 0x1FFF, 0x1FFF),
                                (55, 0x1F, 0x0), (7, 0xF0, 0x30)):
            for n in (0, 5, w - 1, w, w + 1, 2048 + 19, 40001):
                if n < 0:
                    continue
                seed += 1
                out.append((kind, seed, n, 4096, w, mask, target, 100 if mask == 0x3F else 4096, n + 2))
    return out


def run(case):
    kind, seed, n, S, w, mask, target, cS, max_chunks = case
    data = inputs.uniform_unit(seed, 0, n)
    digest = 20 if kind in (SHA1_DIRECT, SHA1_SLIDING) else 16
    out_size = digest if kind in (MD5_DIRECT, SHA1_DIRECT) else oracle.sliding_out_bytes(n, max_chunks, digest)
    st, out = oracle.task(kind, data, out_size, seg_bytes=S, window=w, mask=mask, target=target,
                          chunk_seg_bytes=cS)
    if kind in (MD5_DIRECT, SHA1_DIRECT):
        used, summary = digest, out[:digest].hex()
    else:
        words = (n + 31) // 32
        n_chunks = int.from_bytes(out[0:4], "little")
        flags = int.from_bytes(out[4:8], "little")
        used = 8 + 4 * words + (0 if flags & 1 else (4 + digest) * n_chunks)
        summary = f"chunks={n_chunks}"
    return out_size, st, used, hashlib.sha256(out[:used]).hexdigest(), summary


def main():
    oracle.build()
    lines = ["# CPU-oracle outputs on seeded inputs (written by make_golden.py; see its docstring)",
             "# kind seed n seg_bytes window mask target chunk_seg_bytes out_size status used sha256 summary"]
    for c in cases():
        out_size, st, used, sha, summary = run(c)
        lines.append(" ".join(str(x) for x in (*c[:8], out_size, st, used, sha, summary)))
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(f"{len(lines) - 2} cases -> {OUT}")


if __name__ == "__main__":
    main()
