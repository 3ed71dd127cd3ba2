"""The stored oracle outputs (tests/golden/oracle_cases.txt) still hold.

The file was written from the oracle by tests/golden/make_golden.py; this
test reruns the oracle on every case, and checks the direct cases once more
against hashlib's closed form of direct hashing (an implementation that is
run, never read).  The GPU side is checked against the same file in
test_gpu_parity.py::test_golden_cases_on_gpu."""
import hashlib
import os

import pytest

from paper_1005_1695_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_cases.txt")


def golden_cases():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            rows.append(dict(kind=int(p[0]), seed=int(p[1]), n=int(p[2]), seg=int(p[3]), window=int(p[4]),
                             mask=int(p[5]), target=int(p[6]), cseg=int(p[7]), out_size=int(p[8]),
                             status=int(p[9]), used=int(p[10]), sha=p[11], summary=p[12]))
    return rows


CASES = golden_cases()


def test_golden_file_covers_every_kind():
    assert len(CASES) > 100
    assert {c["kind"] for c in CASES} == {1, 2, 3, 4}


@pytest.mark.parametrize("c", CASES, ids=[f"k{c['kind']}_s{c['seed']}_n{c['n']}" for c in CASES])
def test_oracle_reproduces_golden(oracle_mod, c):
    data = inputs.uniform_unit(c["seed"], 0, c["n"])
    st, out = oracle_mod.task(c["kind"], data, c["out_size"], seg_bytes=c["seg"], window=c["window"],
                              mask=c["mask"], target=c["target"], chunk_seg_bytes=c["cseg"])
    assert st == c["status"]
    assert hashlib.sha256(out[:c["used"]]).hexdigest() == c["sha"]
    if c["kind"] in (1, 3):
        h = hashlib.md5 if c["kind"] == 1 else hashlib.sha1
        x, S = data.tobytes(), c["seg"]
        m = max(1, -(-len(x) // S))
        closed = h(b"".join(h(x[i * S:(i + 1) * S]).digest() for i in range(m))).hexdigest()
        assert c["summary"] == closed
