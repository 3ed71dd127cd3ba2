"""The pins catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of ``oracle/oracle.c`` (a dropped
term, a wrong sign, index, constant or operand order), builds it on the CPU
and runs a fast subset of the pins against it in a child process.  Every
mutant must fail at least one pin; the unmodified copy must pass them all.
"""
import os
import shutil
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

# (name, original text, mutated text)
MUTANTS = [
    ("F_drops_not", "return (x & y) | (~x & z);", "return (x & y) | (x & z);"),
    ("G_drops_not", "return (x & z) | (y & ~z);", "return (x & z) | (y & z);"),
    ("H_drops_term", "return x ^ y ^ z;", "return x ^ y;"),
    ("I_drops_not", "return y ^ (x | ~z);", "return y ^ (x | z);"),
    ("rot_round1", "{7, 12, 17, 22},", "{7, 12, 17, 21},"),
    ("rot_round4", "{6, 10, 15, 21},", "{6, 10, 16, 21},"),
    ("index_round2", "k = (5 * i + 1) % 16;", "k = (5 * i) % 16;"),
    ("index_round3", "k = (3 * i + 5) % 16;", "k = (3 * i + 1) % 16;"),
    ("index_round4", "k = (7 * i) % 16;", "k = (7 * i + 1) % 16;"),
    ("const_index", "T[16 * r + i]", "T[16 * r + (i ^ 1)]"),
    ("rotl_wrong", "static uint32_t rotl32(uint32_t x, int s) { return (x << s) | (x >> (32 - s)); }",
     "static uint32_t rotl32(uint32_t x, int s) { return (x << s) | (x >> (31 - s)); }"),
    ("pad_byte", "tail[rem] = 0x80;", "tail[rem] = 0x01;", "void oracle_md5("),
    ("pad_branch", "(rem < 56) ? 64 : 128", "(rem < 55) ? 64 : 128", "void oracle_md5("),
    ("length_bytes_not_bits", "uint64_t bits = len * 8;", "uint64_t bits = len;", "void oracle_md5("),
    ("sha1_pad_byte", "tail[rem] = 0x80;", "tail[rem] = 0x00;", "void oracle_sha1("),
    ("sha1_pad_branch", "(rem < 56) ? 64 : 128", "(rem <= 56) ? 64 : 128", "void oracle_sha1("),
    ("iv_d", "0x10325476u}", "0x10325477u}"),
    ("out_byte_order", "out[4 * j + 0] = (uint8_t)(st[j]);", "out[4 * j + 0] = (uint8_t)(st[j] >> 24);"),
    ("feed_forward_swap", "st[1] += b;", "st[1] += c;"),
    ("register_rotation", "d = c;\n            c = b;", "d = b;\n            c = c;"),
    ("sin_plus_one", "sin((double)(i + 1))", "sin((double)(i))"),
    ("direct_drops_last_digest", "digest(hash, cat, D * m, out);", "digest(hash, cat, D * (m - 1) + 8, out);"),
    ("direct_empty_zero_segments", "if (n == 0) return 1;", "if (n == 0) return 0;"),
    ("direct_short_segment", "digest(hash, u + off, len, cat + D * i);",
     "digest(hash, u + off, len ? len - 1 : 0, cat + D * i);"),
    ("boundary_sign", "if ((word0 & mask) == target)", "if ((word0 & mask) != target)"),
    ("boundary_big_endian", "uint32_t word0 = (uint32_t)h[0] | ((uint32_t)h[1] << 8)",
     "uint32_t word0 = (uint32_t)h[1] | ((uint32_t)h[0] << 8)"),
    ("last_window_dropped", "for (uint64_t i = 0; i + w <= n; i++) {", "for (uint64_t i = 0; i + w < n; i++) {"),
    ("cut_at_window_start", "uint64_t c = i + w;", "uint64_t c = i + 1;"),
    ("final_cut_duplicated", "if (!(have_last && last == n)) {", "if (1) {"),
    ("chunk_uses_unit_segment_size", "ends[k] - start, chunk_seg_bytes, dig", "ends[k] - start, seg_bytes, dig"),
    ("chunk_start_not_advanced", "            start = ends[k];\n", "\n"),
    ("sha1_schedule_no_rotation", "rotl32s(W[t - 3] ^ W[t - 8] ^ W[t - 14] ^ W[t - 16], 1)",
     "rotl32s(W[t - 3] ^ W[t - 8] ^ W[t - 14] ^ W[t - 16], 0)"),
    ("sha1_maj_as_ch", "else if (t < 60) f = (b & c) ^ (b & d) ^ (c & d);", "else if (t < 60) f = (b & c) ^ (~b & d);"),
    ("sha1_rot30", "c = rotl32s(b, 30);", "c = rotl32s(b, 31);"),
    ("sha1_rot5", "uint32_t T = rotl32s(a, 5) + f + e + K4[t / 20] + W[t];",
     "uint32_t T = rotl32s(a, 5) + f + d + K4[t / 20] + W[t];"),
    ("sha1_const", "0x8f1bbcdcu", "0x8f1bbcddu"),
    ("sha1_iv_e", "0x10325476u, 0xc3d2e1f0u}", "0x10325476u, 0xc3d2e1f1u}"),
    ("sha1_length_little_endian", "tail[tail_len - 1 - j] = (uint8_t)(bits >> (8 * j));",
     "tail[tail_len - 8 + j] = (uint8_t)(bits >> (8 * j));"),
    ("sha1_words_little_endian", "W[t] = ((uint32_t)blk[4 * t] << 24) | ((uint32_t)blk[4 * t + 1] << 16) |",
     "W[t] = ((uint32_t)blk[4 * t + 3] << 24) | ((uint32_t)blk[4 * t + 1] << 16) |"),
    ("sha1_record_size", "uint64_t cap = (out_size - fixed) / (4 + D);", "uint64_t cap = (out_size - fixed) / 20;"),
]

CHECK = textwrap.dedent(
    r"""
    import hashlib, struct, sys
    import numpy as np
    sys.path.insert(0, {root!r})
    import oracle
    oracle.build = lambda force=False: {lib!r}
    from paper_1005_1695_b300 import inputs

    def b(seed, n):
        return inputs.uniform_unit(seed, 7, n).tobytes()

    def direct_cf(x, S):
        m = max(1, -(-len(x) // S))
        return hashlib.md5(b"".join(hashlib.md5(x[i*S:(i+1)*S]).digest() for i in range(m))).digest()

    import mpmath
    mpmath.mp.dps = 50
    assert oracle.md5_table() == [int(mpmath.floor(abs(mpmath.sin(i + 1)) * 2 ** 32)) for i in range(64)]
    for n in list(range(0, 130)) + [4096, 5000]:
        x = b(n, n)
        assert oracle.md5(x) == hashlib.md5(x).digest(), n
    for S in (64, 100):
        for n in (0, 1, S - 1, S, S + 1, 3 * S - 7):
            x = b(n + S, n)
            assert oracle.direct(x, S) == direct_cf(x, S), (n, S)
    for w in (1, 3, 20):
        for mask, target in ((0, 0), (3, 3), (3, 0)):
            for n in range(0, 48):
                x = b(1000 + n, n)
                bits = [i for i in range(0, n - w + 1)
                        if (struct.unpack("<I", hashlib.md5(x[i:i+w]).digest()[:4])[0] & mask) == target]
                bm = oracle.sliding_bitmap(x, w, mask, target)
                want = np.zeros((n + 31) // 32, dtype=np.uint32)
                for i in bits:
                    want[i // 32] |= np.uint32(1 << (i % 32))
                assert np.array_equal(bm, want), (w, mask, n)
                assert list(oracle.chunk_ends(bm, n, w)) == sorted({{i + w for i in bits}} | {{n}})
    n, w, mask, S = 3000, 20, 0x3F, 100
    x = b(2, n)
    bits = [i for i in range(0, n - w + 1)
            if (struct.unpack("<I", hashlib.md5(x[i:i+w]).digest()[:4])[0] & mask) == mask]
    ends = sorted({{i + w for i in bits}} | {{n}})
    st, out = oracle.task(oracle.KIND_MD5_SLIDING, x, oracle.sliding_out_bytes(n, len(ends)),
                          seg_bytes=64, window=w, mask=mask, target=mask, chunk_seg_bytes=S)
    assert st == 0
    cnt, flags, bm, e, dig = oracle.parse_sliding(out, n)
    assert cnt == len(ends) and list(e) == ends
    s = 0
    for k, end in enumerate(ends):
        assert dig[k].tobytes() == direct_cf(x[s:end], S)
        s = end
    for n in list(range(0, 130)) + [4096]:
        x = b(n + 9, n)
        assert oracle.sha1(x) == hashlib.sha1(x).digest(), n
    def sha1_cf(x, S):
        m = max(1, -(-len(x) // S))
        return hashlib.sha1(b"".join(hashlib.sha1(x[i*S:(i+1)*S]).digest() for i in range(m))).digest()
    x = b(5, 3000)
    bits = [i for i in range(0, 3000 - 20 + 1)
            if (struct.unpack("<I", hashlib.sha1(x[i:i+20]).digest()[:4])[0] & 0x3F) == 0x3F]
    ends = sorted({{i + 20 for i in bits}} | {{3000}})
    st, out = oracle.task(oracle.KIND_SHA1_SLIDING, x, oracle.sliding_out_bytes(3000, len(ends), 20),
                          window=20, mask=0x3F, target=0x3F, chunk_seg_bytes=100)
    assert st == 0
    cnt, flags, bm, e, dig = oracle.parse_sliding(out, 3000, 20)
    assert cnt == len(ends) and list(e) == ends
    s0 = 0
    for k, end in enumerate(ends):
        assert dig[k].tobytes() == sha1_cf(x[s0:end], 100)
        s0 = end
    st, out = oracle.task(oracle.KIND_SHA1_SLIDING, x, oracle.sliding_out_bytes(3000, len(ends) - 1, 20),
                          window=20, mask=0x3F, target=0x3F, chunk_seg_bytes=100)
    assert st == 1 and oracle.parse_sliding(out, 3000, 20)[0] == len(ends)
    print("PINS-OK")
    """
)


def _build(src_text, tmp, name):
    c = os.path.join(tmp, name + ".c")
    so = os.path.join(tmp, name + ".so")
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-std=c11", "-O1", "-fPIC", "-shared", c, "-o", so, "-lm"],
                          stderr=subprocess.DEVNULL)
    return so


def _run_pins(lib):
    code = CHECK.format(root=ROOT, lib=lib)
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    return p.returncode == 0 and "PINS-OK" in p.stdout, p


@pytest.fixture(scope="module")
def tmpdir_mod(tmp_path_factory):
    return str(tmp_path_factory.mktemp("mutants"))


def test_unmodified_oracle_passes_subset(tmpdir_mod):
    src = open(SRC).read()
    ok, p = _run_pins(_build(src, tmpdir_mod, "orig"))
    assert ok, p.stdout + p.stderr


def _plant(src, old, new, after=None):
    """Replace the one occurrence of ``old`` (after the marker ``after``, when given)."""
    start = 0
    if after is not None:
        assert src.count(after) == 1, "marker not unique: " + after
        start = src.index(after)
    region = src[start:]
    if after is None:
        assert region.count(old) == 1, "mutation anchor not unique: " + old
    assert old in region, "mutation anchor missing: " + old
    return src[:start] + region.replace(old, new, 1)


@pytest.mark.parametrize("mut", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmpdir_mod, mut):
    name, old, new = mut[:3]
    after = mut[3] if len(mut) > 3 else None
    src = open(SRC).read()
    ok, p = _run_pins(_build(_plant(src, old, new, after), tmpdir_mod, name))
    assert not ok, "mutant survived the pins: " + name
