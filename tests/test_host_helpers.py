"""Host-side helpers of the package that need no GPU: the workload builders
(output sizes, capture slots, the seeded sample the bench checks), the
autotuner's size classes, and the ctypes structures against the header."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def C():
    from paper_1005_1695_b300 import crystal

    crystal.load()
    return crystal


def test_size_classes_boundaries():
    from paper_1005_1695_b300 import autotune as A

    sizes = np.array([0, 1, (64 << 10) - 1, 64 << 10, (1 << 20) - 1, 1 << 20, 64 << 20])
    assert A.size_classes(sizes).tolist() == [0, 0, 0, 1, 1, 2, 2]


def test_out_sizes_and_capture_slots(C):
    from paper_1005_1695_b300 import streams as S

    req, cap = S.make_trace(9, 400, 5000.0, 256 << 20, capture_every=3)
    for r in req:
        k, n = int(r["kind"]), int(r["size"])
        if k in C.SLIDING_KINDS:
            assert int(r["out_size"]) == C.sliding_out_bytes(n, 4 * (n // 8192) + 64, k)
            assert int(r["out_size"]) >= 8 + 4 * ((n + 31) // 32)
        else:
            assert int(r["out_size"]) == C.digest_size(k)
    slots = [(int(r["capture_offset"]), int(r["out_size"])) for r in req if int(r["capture_offset"]) != C.NO_CAPTURE]
    assert len(slots) == (len(req) + 2) // 3
    end = 0
    for off, size in slots:  # 16-byte aligned, in order, no overlap, inside the buffer
        assert off % 16 == 0 and off >= end
        end = off + size
    assert end <= cap
    # a SHA-1 sliding request gets 24-byte records
    req["kind"][0] = C.CRYSTAL_KIND_SHA1_SLIDING
    S.set_out_sizes(req)
    n0 = int(req["size"][0])
    assert int(req["out_size"][0]) == 8 + 4 * ((n0 + 31) // 32) + 24 * (4 * (n0 // 8192) + 64)


def test_bench_sample_keeps_largest_units(C):
    import bench

    from paper_1005_1695_b300 import streams as S

    req, _ = S.make_batch(11, 5000, 1 << 30)
    idx = bench._sample(req["size"], req["kind"], 100)
    assert len(idx) >= 50 and idx == sorted(set(idx))
    for group in (C.DIRECT_KINDS, C.SLIDING_KINDS):
        sizes = [int(req["size"][i]) for i in range(len(req)) if int(req["kind"][i]) in group]
        chosen = [int(req["size"][i]) for i in idx if int(req["kind"][i]) in group]
        assert max(sizes) == max(chosen)


def test_geometry_and_stream_structs_match_header(C):
    import ctypes

    assert ctypes.sizeof(C.crystal_geometry) == 24
    assert ctypes.sizeof(C.crystal_stream_config) == 32
    assert ctypes.sizeof(C.crystal_serve_config) == 64
    g = C.geometry(seg_threads=64, win_registers=64)
    assert g.as_dict()["seg_threads"] == 64 and g.reserved == 0


def test_ctypes_layouts_match_the_c_compiler(C, tmp_path):
    """Every structure the binding mirrors, sized and laid out by gcc from
    include/crystal.h, against its ctypes / numpy twin."""
    import ctypes
    import os
    import subprocess

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "sizes.c"
    src.write_text('''#include <stdio.h>
#include <stddef.h>
#include "crystal.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(crystal_config), sizeof(crystal_hash_params),
         sizeof(crystal_stats), sizeof(crystal_unit), sizeof(crystal_batch), sizeof(crystal_request),
         sizeof(crystal_request_result), sizeof(crystal_serve_config), sizeof(crystal_stream_config),
         sizeof(crystal_geometry), offsetof(crystal_serve_config, bypass_ns),
         offsetof(crystal_serve_config, ring_max_request));
  return 0;
}
''')
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(C.crystal_config), ctypes.sizeof(C.crystal_hash_params), ctypes.sizeof(C.crystal_stats),
            C.UNIT_DTYPE.itemsize, C.BATCH_HEADER_BYTES, C.REQUEST_DTYPE.itemsize, C.RESULT_DTYPE.itemsize,
            ctypes.sizeof(C.crystal_serve_config), ctypes.sizeof(C.crystal_stream_config),
            ctypes.sizeof(C.crystal_geometry), C.crystal_serve_config.bypass_ns.offset,
            C.crystal_serve_config.ring_max_request.offset]
    assert got == want
