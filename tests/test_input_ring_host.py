"""The serving loop's input ring (``csrc/input_ring.h``), host logic only:
compiled with g++ into a small driver and run under random take / give-back
churn.  Checked against properties that do not depend on the placement
policy (live slots never overlap and stay inside the ring, 256-byte aligned,
every slot reclaimed in the end, an empty ring always grants a slot that
fits) and against a plain model of the policy (a slot goes right after the
newest live slot, or to the start when the end is reached and the oldest
live slot leaves room; finished slots are reclaimed oldest first)."""
import os
import random
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1005_1695_b300", "csrc")
NONE = (1 << 64) - 1

DRIVER = r"""
#include <stdio.h>
#include "input_ring.h"
int main(void) {
  unsigned long long bytes;
  if (scanf("%llu", &bytes) != 1) return 2;
  crystal::InputRing r;
  r.init(bytes);
  char op;
  unsigned long long v;
  while (scanf(" %c %llu", &op, &v) == 2) {
    if (op == 't') {
      uint64_t seq = 0;
      const uint64_t off = r.take(v, &seq);
      if (off == crystal::InputRing::kNone) printf("none\n");
      else printf("%llu %llu\n", (unsigned long long)off, (unsigned long long)seq);
    } else if (op == 'g') {
      r.give_back(v);
      printf("ok\n");
    } else if (op == 'n') {
      printf("%llu\n", (unsigned long long)r.live_slots());
    }
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    d = tmp_path_factory.mktemp("ring")
    src = d / "ring.cpp"
    src.write_text(DRIVER)
    exe = d / "ring"
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe), "-lpthread"])
    return str(exe)


def run(driver, ring_bytes, ops):
    text = "%d\n" % ring_bytes + "".join("%s %d\n" % op for op in ops)
    out = subprocess.run([driver], input=text.encode(), stdout=subprocess.PIPE, check=True).stdout.decode()
    return out.split("\n")[:len(ops)]


class Model:
    """The policy written out plainly: live slots oldest first as
    [seq, off, len, done]."""

    def __init__(self, size):
        self.size, self.live, self.front = size, [], 0

    def take(self, n):
        b = ((n or 1) + 255) // 256 * 256
        if not self.live:
            off = 0 if b <= self.size else None
        else:
            first = self.live[0][1]
            end = self.live[-1][1] + self.live[-1][2]
            if self.live[-1][1] >= first:
                off = end if end + b <= self.size else (0 if b <= first else None)
            else:
                off = end if end + b <= first else None
        if off is None:
            return None
        seq = self.front + len(self.live)
        self.live.append([seq, off, b, False])
        return off, seq

    def give(self, seq):
        k = seq - self.front
        if k < 0 or k >= len(self.live):
            return
        if k == len(self.live) - 1 and len(self.live) > 1:
            self.live.pop()
            return
        self.live[k][3] = True
        while self.live and self.live[0][3]:
            self.live.pop(0)
            self.front += 1


@pytest.mark.parametrize("seed", range(6))
def test_ring_under_churn_matches_policy_and_never_overlaps(driver, seed):
    rng = random.Random(seed)
    ring_bytes = rng.choice([4096, 1 << 16, 3 << 20])
    ops, expect, held = [], [], []
    model = Model(ring_bytes)
    for _ in range(3000):
        if held and (rng.random() < 0.45 or len(held) > 40):
            # completions out of order: any held slot may finish
            seq = held.pop(rng.randrange(len(held)))
            ops.append(("g", seq))
            model.give(seq)
            expect.append(("ok",))
        else:
            n = rng.choice([0, 1, 255, 256, 257, rng.randrange(1, ring_bytes // 3 + 2)])
            ops.append(("t", n))
            got = model.take(n)
            expect.append(got)
            if got is not None:
                held.append(got[1])
    lines = run(driver, ring_bytes, ops)
    live = {}  # seq -> (off, len) of slots handed out and not yet given back
    for op, line, want in zip(ops, lines, expect):
        if op[0] == "t":
            if want is None:
                assert line == "none"
                continue
            off, seq = (int(x) for x in line.split())
            assert (off, seq) == want
            b = ((op[1] or 1) + 255) // 256 * 256
            assert off % 256 == 0 and off + b <= ring_bytes
            for o2, b2 in live.values():
                assert off + b <= o2 or o2 + b2 <= off, "overlapping live slots"
            live[seq] = (off, b)
        else:
            assert line == "ok"
            live.pop(op[1])


def test_ring_reclaims_everything_and_grants_when_empty(driver):
    ops = [("t", 5000), ("t", 70000), ("t", 100), ("g", 1), ("g", 0), ("g", 2), ("n", 0),
           ("t", 1 << 20), ("g", 3), ("n", 0), ("t", (1 << 20) + 1)]
    lines = run(driver, 1 << 20, ops)
    assert lines[0] == "0 0" and lines[1] == "5120 1" and lines[2] == "75264 2"
    assert lines[6] == "0"                        # every slot reclaimed
    assert lines[7].split()[0] == "0"             # an empty ring grants a slot as large as itself at 0
    assert lines[9] == "0" and lines[10] == "none"  # larger than the ring: never


def test_ring_refuses_sizes_that_would_wrap(driver):
    lines = run(driver, 1 << 20, [("t", (1 << 64) - 1), ("t", (1 << 64) - 200), ("n", 0), ("t", 100)])
    assert lines[:3] == ["none", "none", "0"] and lines[3] == "0 0"


def test_ring_wraps_and_waits_for_the_oldest(driver):
    R = 4096
    ops = [("t", 1024), ("t", 1024), ("t", 1024), ("t", 1024),  # full: seqs 0-3 at 0,1024,2048,3072
           ("t", 1),                                             # no room
           ("g", 1), ("t", 1024),                                # slot 1 done, but 0 is older: still none
           ("g", 0), ("t", 2048),                                # 0 and 1 reclaimed: wrap to 0
           ("t", 256)]                                           # wrapped, gap [2048, 2048): none
    lines = run(driver, R, ops)
    assert lines[4] == "none" and lines[6] == "none"
    assert lines[8] == "0 4" and lines[9] == "none"
