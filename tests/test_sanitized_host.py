"""Host-side structures of the runtime built with sanitizers and stressed on
the CPU (no GPU): the arena allocator and batch planner (``csrc/plan.cpp``)
and the serving loop's input ring (``csrc/input_ring.h``) under
AddressSanitizer + UndefinedBehaviorSanitizer, and both again under
ThreadSanitizer with several threads allocating and freeing at once, as the
admission loop, the copy threads and the master thread do.  A sanitizer
report fails the test (every error aborts the driver)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1005_1695_b300", "csrc")
INCLUDE = os.path.join(ROOT, "include")
CUDA_INCLUDE = "/usr/local/cuda/include"

DRIVER = r"""
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <random>
#include <thread>
#include <vector>

#include "crystal.h"
#include "crystal_internal.h"
#include "input_ring.h"

#define CHECK(c) do { if (!(c)) { fprintf(stderr, "check failed: %s (line %d)\n", #c, __LINE__); abort(); } } while (0)

// Arena: random allocations at both ends, exact placements and frees, with
// the live blocks' bytes recounted against crystal_arena_used.
static void arena_churn(crystal_arena* a, uint64_t size, unsigned seed, int rounds, bool check_used) {
    std::mt19937_64 rng(seed);
    std::vector<std::pair<uint64_t, uint64_t>> live;  // offset, bytes asked
    for (int r = 0; r < rounds; ++r) {
        const unsigned op = rng() % 10;
        if (op < 5 || live.empty()) {
            const uint64_t n = 1 + rng() % (size / 16);
            uint64_t off = 0;
            const int placement = (op & 1) ? CRYSTAL_ARENA_LOWEST : CRYSTAL_ARENA_HIGHEST;
            if (crystal_arena_alloc_at(a, n, placement, &off) == CRYSTAL_OK) {
                CHECK(off % 256 == 0 && off + n <= size);
                live.push_back({off, n});
            }
        } else if (op == 5) {
            const uint64_t n = 1 + rng() % (size / 64);
            const uint64_t off = (rng() % (size / 256)) * 256;
            if (off + n <= size && crystal_arena_alloc_exact(a, off, n) == CRYSTAL_OK) live.push_back({off, n});
        } else {
            const size_t k = rng() % live.size();
            CHECK(crystal_arena_free(a, live[k].first) == CRYSTAL_OK);
            live[k] = live.back();
            live.pop_back();
        }
        if (check_used && r % 64 == 0) {
            uint64_t sum = 0;
            for (auto& b : live) sum += (b.second + 255) / 256 * 256;
            CHECK(crystal_arena_used(a) == sum);
        }
    }
    for (auto& b : live) CHECK(crystal_arena_free(a, b.first) == CRYSTAL_OK);
}

// Batch planner on random descriptors (direct units first, then sliding).
static void plan_churn(unsigned seed, int rounds) {
    std::mt19937_64 rng(seed);
    for (int r = 0; r < rounds; ++r) {
        const uint32_t nd = rng() % 9, ns = rng() % 9;
        std::vector<uint8_t> mem(crystal_batch_bytes(nd + ns));
        crystal_batch* b = reinterpret_cast<crystal_batch*>(mem.data());
        crystal_unit* u = crystal::batch_units(b);
        for (uint32_t i = 0; i < nd + ns; ++i) {
            const bool sliding = i >= nd;
            const uint64_t n = rng() % (1u << 20);
            u[i].in = 0x100000 + 16 * i;
            u[i].n = n;
            u[i].out = 0x900000 + 4096 * i;
            u[i].scratch = 0x1900000 + 65536 * i;
            u[i].seg_bytes = 1 + rng() % 65536;
            u[i].kind = sliding ? ((rng() & 1) ? CRYSTAL_KIND_SHA1_SLIDING : CRYSTAL_KIND_MD5_SLIDING)
                                : ((rng() & 1) ? CRYSTAL_KIND_SHA1_DIRECT : CRYSTAL_KIND_MD5_DIRECT);
            u[i].window = sliding ? 1 + rng() % 55 : 0;
            u[i].mask = 0x1FFF;
            u[i].target = 0x1FFF;
            u[i].out_cap = sliding ? (uint32_t)crystal_sliding_out_bytes(n, 64) : 20;
        }
        const int st = crystal_batch_plan(b, nd, ns);
        CHECK(st == CRYSTAL_OK || st == CRYSTAL_EINVAL);
    }
}

// Input ring: slots taken in one order and given back in another, checked
// never to overlap.
static void ring_churn(unsigned seed, int rounds) {
    crystal::InputRing ring;
    const uint64_t size = 1 << 20;
    ring.init(size);
    std::mt19937_64 rng(seed);
    struct Slot { uint64_t off, len, seq; };
    std::vector<Slot> held;
    for (int r = 0; r < rounds; ++r) {
        if (!held.empty() && (rng() % 2 || held.size() > 50)) {
            const size_t k = rng() % held.size();
            ring.give_back(held[k].seq);
            held[k] = held.back();
            held.pop_back();
        } else {
            const uint64_t n = rng() % (size / 5);
            uint64_t seq = 0;
            const uint64_t off = ring.take(n, &seq);
            if (off == crystal::InputRing::kNone) continue;
            const uint64_t len = (n ? n : 1) + 255 & ~(uint64_t)255;
            CHECK(off + len <= size);
            for (auto& h : held) CHECK(off + len <= h.off || h.off + h.len <= off);
            held.push_back({off, len, seq});
        }
    }
    for (auto& h : held) ring.give_back(h.seq);
    CHECK(ring.live_slots() == 0);
}

// Threads at once: each takes arena blocks and ring slots and frees them,
// some freed by another thread (as completions free what admission took).
static void threaded(crystal_arena* a) {
    crystal::InputRing ring;
    ring.init(4 << 20);
    std::mutex mu;
    std::vector<uint64_t> handoff_arena, handoff_ring;
    std::atomic<bool> done{false};
    std::vector<std::thread> th;
    for (int t = 0; t < 4; ++t) {
        th.emplace_back([&, t] {
            std::mt19937_64 rng(100 + t);
            for (int r = 0; r < 4000; ++r) {
                uint64_t off = 0, seq = 0;
                if (crystal_arena_alloc_at(a, 1 + rng() % 65536, (r & 1) ? CRYSTAL_ARENA_LOWEST : CRYSTAL_ARENA_HIGHEST,
                                           &off) == CRYSTAL_OK) {
                    std::lock_guard<std::mutex> lk(mu);
                    handoff_arena.push_back(off);
                }
                if (ring.take(rng() % 70000, &seq) != crystal::InputRing::kNone) {
                    std::lock_guard<std::mutex> lk(mu);
                    handoff_ring.push_back(seq);
                }
            }
        });
    }
    std::thread freer([&] {
        for (;;) {
            std::vector<uint64_t> fa, fr;
            {
                std::lock_guard<std::mutex> lk(mu);
                fa.swap(handoff_arena);
                fr.swap(handoff_ring);
            }
            for (uint64_t off : fa) CHECK(crystal_arena_free(a, off) == CRYSTAL_OK);
            for (uint64_t s : fr) ring.give_back(s);
            if (fa.empty() && fr.empty() && done.load()) break;
            std::this_thread::yield();
        }
    });
    for (auto& x : th) x.join();
    done.store(true);
    freer.join();
    CHECK(crystal_arena_used(a) == 0);
    CHECK(ring.live_slots() == 0);
}

int main(int argc, char** argv) {
    const bool threads_only = argc > 1 && !strcmp(argv[1], "threads");
    crystal_arena* a = nullptr;
    const uint64_t size = 64ull << 20;
    CHECK(crystal_arena_create(size, 256, &a) == CRYSTAL_OK);
    if (!threads_only) {
        arena_churn(a, size, 1, 20000, true);
        CHECK(crystal_arena_used(a) == 0);
        plan_churn(2, 3000);
        ring_churn(3, 20000);
    }
    threaded(a);
    crystal_arena_destroy(a);
    printf("ok\n");
    return 0;
}
"""


def _build(tmp_path, name, flags):
    src = tmp_path / "driver.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / name
    cmd = ["g++", "-std=c++17", "-g", "-O1", "-fno-omit-frame-pointer", *flags, "-I", INCLUDE, "-I", CSRC,
           "-I", CUDA_INCLUDE, str(src), os.path.join(CSRC, "plan.cpp"), "-o", str(exe), "-lpthread"]
    subprocess.check_call(cmd)
    return str(exe)


needs_tools = pytest.mark.skipif(shutil.which("g++") is None or not os.path.isdir(CUDA_INCLUDE),
                                 reason="g++ and the CUDA headers are needed to build the host driver")


@needs_tools
def test_arena_planner_ring_under_address_and_ub_sanitizers(tmp_path):
    exe = _build(tmp_path, "asan", ["-fsanitize=address,undefined", "-fno-sanitize-recover=all"])
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([exe], env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == b"ok", r.stderr.decode()[-4000:]


@needs_tools
def test_arena_and_ring_threads_under_thread_sanitizer(tmp_path):
    exe = _build(tmp_path, "tsan", ["-fsanitize=thread"])
    env = dict(os.environ, TSAN_OPTIONS="halt_on_error=1:exitcode=66")
    r = subprocess.run([exe, "threads"], env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == b"ok", r.stderr.decode()[-4000:]
