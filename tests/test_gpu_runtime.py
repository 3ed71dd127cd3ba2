"""The job runtime (pool, streams, master thread, callbacks) on the GPU.

Every job's output is compared bit for bit with the CPU oracle; the runtime
modes (pooled / per-job allocation, overlap / sequential, batched / one job
per launch, graphs) must all give the same bytes, and a job's result must be
the same alone and in a mix.  Failure paths are driven from the host: a
full pool, a too-small output buffer, a bounded wait that runs out, an
allocation that cannot succeed at init, shutdown with jobs in flight.
"""
import ctypes
import threading

import numpy as np
import pytest

from helpers import first_difference, same_result

pytestmark = pytest.mark.gpu

DIRECT, SLIDING, NOP = 1, 2, 0
SEC = 1_000_000_000


@pytest.fixture(scope="module")
def C():
    import torch

    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    from paper_1005_1695_b300 import crystal

    crystal.load()
    return crystal


def _jobs(C, count=24, seed=7):
    from paper_1005_1695_b300 import inputs

    jobs = []
    for i in range(count):
        n = int([65536, 1 << 20, 4097, 0, 300000, 20][i % 6]) + (i % 5) * 3
        if i % 3 == 1:
            data = inputs.dedup_unit(seed, i, n)
            p = C.params(mask=0x3FF, target=0x3FF)
            jobs.append((SLIDING, data, C.sliding_out_bytes(n, n // 256 + 16), p))
        else:
            data = inputs.uniform_unit(seed, i, n)
            p = C.params(segment_bytes=[4096, 1024, 333][i % 3])
            jobs.append((DIRECT, data, 16, p))
    return jobs


def _want(oracle_mod, jobs):
    out = []
    for kind, data, osz, p in jobs:
        st, w = oracle_mod.task(kind, data, osz, seg_bytes=p.segment_bytes, window=p.window_bytes,
                                mask=p.mask, target=p.target, chunk_seg_bytes=p.chunk_segment_bytes)
        out.append((st, w))
    return out


def _submit_all(C, ctx, jobs, callback=None):
    tasks = []
    for kind, data, osz, p in jobs:
        t = ctx.task_create(len(data), osz)
        t.h_in[:] = data
        assert t.submit(kind, p, callback) == C.CRYSTAL_OK
        tasks.append(t)
    return tasks


def _check(C, tasks, jobs, want):
    for i, (t, (kind, data, osz, p), (ost, w)) in enumerate(zip(tasks, jobs, want)):
        st = t.wait(30 * SEC)
        assert st == (C.CRYSTAL_OK if ost == 0 else C.CRYSTAL_EOVERFLOW), (i, st)
        g = t.output()
        assert same_result(kind, len(data), g, w), f"job {i}: " + first_difference(kind, len(data), g, w)


@pytest.mark.parametrize("flags", [0, 1, 2, 4, 8, 1 | 2 | 4], ids=["pooled", "no_pool", "no_overlap", "no_batch",
                                                                  "graphs", "plain"])
def test_runtime_modes_bit_exact(C, oracle_mod, flags):
    jobs = _jobs(C)
    want = _want(oracle_mod, jobs)
    with C.Context(max_in_bytes=2 << 20, max_out_bytes=1 << 20, device_pool_bytes=256 << 20,
                   host_pool_bytes=128 << 20, n_streams=3, flags=flags, max_batch_jobs=8) as ctx:
        used0 = ctx.stats().device_pool_used
        tasks = _submit_all(C, ctx, jobs)
        _check(C, tasks, jobs, want)
        s = ctx.stats()
        assert s.jobs_completed == len(jobs)
        for t in tasks:
            assert t.release() == C.CRYSTAL_OK
        after = ctx.stats()
        assert after.device_pool_used == used0 and after.host_pool_used == 0


def test_prepared_graphs_are_replayed_not_captured(C, oracle_mod):
    """crystal_prepare_graphs captures every stream slot's graph for every
    batch size class and kind mix up front; a mixed stream afterwards
    captures nothing and stays bit-exact.  Without graphs it does nothing."""
    jobs = _jobs(C)
    want = _want(oracle_mod, jobs)
    with C.Context(max_in_bytes=2 << 20, max_out_bytes=1 << 20, device_pool_bytes=256 << 20,
                   host_pool_bytes=128 << 20, n_streams=3, flags=C.CRYSTAL_FLAG_GRAPHS, max_batch_jobs=8) as ctx:
        assert ctx.stats().graph_captures == 0
        ctx.prepare_graphs()
        n = ctx.stats().graph_captures
        assert n == 3 * 2 * C.CRYSTAL_SIZE_CLASSES * 3  # slots x size classes x kind mixes
        ctx.prepare_graphs()  # nothing left to capture
        assert ctx.stats().graph_captures == n
        tasks = _submit_all(C, ctx, jobs)
        _check(C, tasks, jobs, want)
        assert ctx.stats().graph_captures == n
        for t in tasks:
            t.release()
        # a geometry change drops that class's graphs; preparing again recaptures them
        ctx.set_geometry(1, C.geometry(seg_threads=64))
        ctx.prepare_graphs()
        assert ctx.stats().graph_captures == n + 3 * 2 * 3
    with C.Context(max_in_bytes=1 << 20, max_out_bytes=1 << 16, device_pool_bytes=64 << 20,
                   host_pool_bytes=64 << 20, n_streams=2) as ctx:
        ctx.prepare_graphs()
        assert ctx.stats().graph_captures == 0


def test_application_threads_share_one_context(C, oracle_mod):
    """Eight application threads create, fill, submit, wait for and release
    jobs on one context at the same time (some waiting job by job, some with
    wait_many), over many rounds with a small pool, so creation meets EAGAIN
    while other threads free room: every output bit-exact, the pools whole at
    the end."""
    jobs = _jobs(C, count=24, seed=21)
    want = _want(oracle_mod, jobs)
    errors = []
    with C.Context(max_in_bytes=2 << 20, max_out_bytes=1 << 20, device_pool_bytes=8 << 20,
                   host_pool_bytes=8 << 20, n_streams=4, max_batch_jobs=8, flags=C.CRYSTAL_FLAG_GRAPHS) as ctx:
        used0 = ctx.stats().device_pool_used

        def worker(k):
            held = []

            def drain():
                if k % 2 and held:
                    ctx.wait_many([t for _, t in held], 60 * SEC)
                for i, t in held:
                    kind, data = jobs[i][0], jobs[i][1]
                    st = t.wait(60 * SEC)
                    assert st == (C.CRYSTAL_OK if want[i][0] == 0 else C.CRYSTAL_EOVERFLOW), (k, i, st)
                    assert same_result(kind, len(data), t.output(), want[i][1]), (k, i)
                    assert t.release() == C.CRYSTAL_OK
                held.clear()

            try:
                for r in range(6):
                    for i in [i for i in range(len(jobs)) if (i + k + r) % 8 == 0]:
                        kind, data, osz, p = jobs[i]
                        for attempt in range(20000):  # bounded: ~10 s of retries at most
                            try:
                                t = ctx.task_create(len(data), osz)
                                break
                            except C.CrystalError as e:
                                # pool full: finish this thread's own jobs (never
                                # hold buffers while waiting for room), then retry
                                assert e.status == C.CRYSTAL_EAGAIN, e
                                drain()
                                threading.Event().wait(0.0005)
                        else:
                            raise AssertionError("no room for a job after 20,000 tries")
                        t.h_in[:] = data
                        assert t.submit(kind, p) == C.CRYSTAL_OK
                        held.append((i, t))
                    drain()
            except Exception as e:  # reported on the main thread
                errors.append(e)

        threads = [threading.Thread(target=worker, args=(k,)) for k in range(8)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        assert not errors, errors[0]
        s = ctx.stats()
        assert s.device_pool_used == used0 and s.host_pool_used == 0
        assert s.jobs_completed == 6 * len(jobs)


def test_graph_preparation_and_geometry_refused_while_busy(C, oracle_mod):
    """While a job is running (its callback is held open, so the master has
    not retired it), crystal_prepare_graphs and crystal_set_geometry refuse
    with EINVAL and change nothing; once the job is retired both succeed, and
    the job's output is exact."""
    jobs = _jobs(C, count=1, seed=31)
    want = _want(oracle_mod, jobs)
    entered, gate = threading.Event(), threading.Event()

    @C.crystal_callback
    def cb(handle, status, user):
        entered.set()
        gate.wait(20)  # bounded: the test sets it at once

    with C.Context(max_in_bytes=2 << 20, max_out_bytes=1 << 20, device_pool_bytes=64 << 20,
                   host_pool_bytes=64 << 20, n_streams=2, flags=C.CRYSTAL_FLAG_GRAPHS) as ctx:
        kind, data, osz, p = jobs[0]
        t = ctx.task_create(len(data), osz)
        t.h_in[:] = data
        assert t.submit(kind, p, cb) == C.CRYSTAL_OK
        assert entered.wait(30)
        try:
            captures = ctx.stats().graph_captures
            L = C.load()
            assert L.crystal_prepare_graphs(ctx.handle) == C.CRYSTAL_EINVAL
            g = C.geometry(seg_threads=64)
            assert L.crystal_set_geometry(ctx.handle, 0, ctypes.byref(g)) == C.CRYSTAL_EINVAL
            assert ctx.stats().graph_captures == captures
        finally:
            gate.set()
        assert t.wait(30 * SEC) == (C.CRYSTAL_OK if want[0][0] == 0 else C.CRYSTAL_EOVERFLOW)
        assert same_result(kind, len(data), t.output(), want[0][1])
        assert t.release() == C.CRYSTAL_OK
        ctx.set_geometry(0, C.geometry(seg_threads=64))
        ctx.prepare_graphs()
        assert ctx.stats().graph_captures > captures


def test_resubmit_reuses_buffers(C, oracle_mod):
    jobs = _jobs(C, count=6, seed=11)
    want = _want(oracle_mod, jobs)
    with C.Context(max_in_bytes=2 << 20, max_out_bytes=1 << 20, device_pool_bytes=64 << 20,
                   host_pool_bytes=64 << 20) as ctx:
        t = ctx.task_create(2 << 20, 1 << 20)
        for (kind, data, osz, p), (ost, w) in zip(jobs, want):
            t.resize(len(data), osz)
            t.h_in[:len(data)] = data
            assert t.submit(kind, p) == C.CRYSTAL_OK
            assert t.wait(30 * SEC) == (C.CRYSTAL_OK if ost == 0 else C.CRYSTAL_EOVERFLOW)
            assert same_result(kind, len(data), t.output(), w)
        assert t.release() == C.CRYSTAL_OK


def test_alone_equals_in_mix(C, oracle_mod):
    jobs = _jobs(C, count=18, seed=13)
    with C.Context(max_in_bytes=2 << 20, max_out_bytes=1 << 20, device_pool_bytes=256 << 20,
                   host_pool_bytes=128 << 20, n_streams=4, max_batch_jobs=16) as ctx:
        alone = []
        for job in jobs:
            t = _submit_all(C, ctx, [job])[0]
            t.wait(30 * SEC)
            alone.append(t.output())
            t.release()
        tasks = _submit_all(C, ctx, jobs)
        for i, t in enumerate(tasks):
            t.wait(30 * SEC)
            kind, data = jobs[i][0], jobs[i][1]
            assert same_result(kind, len(data), t.output(), alone[i]), i


def test_callbacks_fire_once_and_may_release(C, oracle_mod):
    jobs = _jobs(C, count=12, seed=17)
    want = _want(oracle_mod, jobs)
    seen = {}
    lock = threading.Lock()
    done = threading.Event()
    L = C.load()

    @C.crystal_callback
    def cb(handle, status, user):
        with lock:
            seen[handle] = seen.get(handle, []) + [status]
            if len(seen) == len(jobs):
                done.set()

    with C.Context(max_in_bytes=2 << 20, max_out_bytes=1 << 20, device_pool_bytes=128 << 20,
                   host_pool_bytes=64 << 20) as ctx:
        tasks = _submit_all(C, ctx, jobs, callback=cb)
        assert done.wait(30)
        for t, (ost, _) in zip(tasks, want):
            assert seen[t.handle] == [C.CRYSTAL_OK if ost == 0 else C.CRYSTAL_EOVERFLOW]
        used_before = ctx.stats().host_pool_used

        # a callback that releases its own job
        released = threading.Event()

        @C.crystal_callback
        def cb_release(handle, status, user):
            assert L.crystal_task_wait(handle, 0) == C.CRYSTAL_EINVAL  # no waiting inside a callback
            assert L.crystal_task_release(handle) == C.CRYSTAL_OK
            released.set()

        t = ctx.task_create(4096, 16)
        t.h_in[:] = 1
        assert t.submit(DIRECT, None, cb_release) == C.CRYSTAL_OK
        assert released.wait(30)
        ctx._tasks.discard(t)
        import time

        for _ in range(100):
            if ctx.stats().host_pool_used == used_before:
                break
            time.sleep(0.01)
        assert ctx.stats().host_pool_used == used_before


def test_overflow_status_through_runtime(C, oracle_mod):
    from paper_1005_1695_b300 import inputs

    n = 50000
    data = inputs.uniform_unit(3, 3, n)
    p = C.params(mask=0x3, target=0x3)
    with C.Context(max_in_bytes=1 << 20, max_out_bytes=1 << 20, device_pool_bytes=64 << 20,
                   host_pool_bytes=32 << 20) as ctx:
        osz = C.sliding_out_bytes(n, 100)
        t = ctx.task_create(n, osz)
        t.h_in[:] = data
        assert t.submit(SLIDING, p) == C.CRYSTAL_OK
        assert t.wait(30 * SEC) == C.CRYSTAL_EOVERFLOW
        st, w = oracle_mod.task(SLIDING, data, osz, mask=0x3, target=0x3)
        assert st == 1 and same_result(SLIDING, n, t.output(), w)


def test_pool_exhaustion_is_eagain_then_recovers(C):
    with C.Context(max_in_bytes=8 << 20, max_out_bytes=1 << 20, device_pool_bytes=32 << 20,
                   host_pool_bytes=32 << 20) as ctx:
        held = []
        with pytest.raises(C.CrystalError) as e:
            for _ in range(64):
                held.append(ctx.task_create(4 << 20, 16))
        assert e.value.status == C.CRYSTAL_EAGAIN
        assert 1 <= len(held) < 64
        held.pop().release()
        t = ctx.task_create(4 << 20, 16)
        t.h_in[:] = 5
        assert t.submit(DIRECT) in (C.CRYSTAL_OK, C.CRYSTAL_EAGAIN)


def test_bad_arguments_are_rejected(C):
    with C.Context(max_in_bytes=1 << 20, max_out_bytes=1 << 20, device_pool_bytes=16 << 20,
                   host_pool_bytes=16 << 20) as ctx:
        with pytest.raises(C.CrystalError):
            ctx.task_create(2 << 20, 16)  # above max_in_bytes
        t = ctx.task_create(1000, 8)
        assert t.submit(DIRECT) == C.CRYSTAL_EINVAL  # out < 16
        assert t.submit(SLIDING) == C.CRYSTAL_EINVAL  # out < header + bitmap
        assert t.submit(7) == C.CRYSTAL_EINVAL
        t2 = ctx.task_create(1000, 4096)
        assert t2.submit(SLIDING, C.params(window_bytes=56)) == C.CRYSTAL_EINVAL
        assert t2.poll() == C.CRYSTAL_EINVAL  # never submitted
        assert t2.wait(0) == C.CRYSTAL_EINVAL


def test_wait_timeout_then_completes(C):
    with C.Context(max_in_bytes=64 << 20, max_out_bytes=8 << 20, device_pool_bytes=512 << 20,
                   host_pool_bytes=256 << 20) as ctx:
        n = 48 << 20
        t = ctx.task_create(n, C.sliding_out_bytes(n, 1 << 14))
        t.h_in[:] = 7
        assert t.submit(SLIDING) == C.CRYSTAL_OK
        assert t.wait(0) == C.CRYSTAL_ETIMEDOUT
        assert t.poll() in (C.CRYSTAL_PENDING, C.CRYSTAL_OK)
        assert t.wait(60 * SEC) == C.CRYSTAL_OK
        assert t.poll() == C.CRYSTAL_OK


def test_init_allocation_failure_is_clean(C):
    with pytest.raises(RuntimeError):
        C.Context(device_pool_bytes=1 << 50)
    with pytest.raises(RuntimeError):
        C.Context(n_streams=0 - 1)
    with C.Context(device_pool_bytes=16 << 20, host_pool_bytes=16 << 20) as ctx:  # still usable
        t = ctx.task_create(100, 16)
        t.h_in[:] = 0
        assert t.submit(DIRECT) == 0 and t.wait(10 * SEC) == 0


def test_shutdown_with_jobs_in_flight(C):
    ctx = C.Context(max_in_bytes=4 << 20, max_out_bytes=1 << 20, device_pool_bytes=256 << 20,
                    host_pool_bytes=128 << 20, n_streams=2, max_batch_jobs=2)
    statuses = []

    @C.crystal_callback
    def cb(handle, status, user):
        statuses.append(status)

    for i in range(20):
        t = ctx.task_create(4 << 20, 16)
        t.h_in[:] = i
        assert t.submit(DIRECT, None, cb) == C.CRYSTAL_OK
    assert ctx.shutdown() == C.CRYSTAL_OK
    assert len(statuses) == 20
    assert set(statuses) <= {C.CRYSTAL_OK, C.CRYSTAL_ESHUTDOWN}


def test_nop_jobs_copy_through(C):
    with C.Context(max_in_bytes=1 << 20, max_out_bytes=1 << 20, device_pool_bytes=16 << 20,
                   host_pool_bytes=16 << 20) as ctx:
        t = ctx.task_create(4096, 4096)
        t.h_in[:] = 3
        assert t.submit(NOP) == C.CRYSTAL_OK
        assert t.wait(10 * SEC) == C.CRYSTAL_OK
        s, d, e = t.timing()
        assert 0 < s <= d <= e


def test_external_device_arena(C, oracle_mod):
    import torch

    arena = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    jobs = _jobs(C, count=6, seed=23)
    want = _want(oracle_mod, jobs)
    with C.Context(max_in_bytes=2 << 20, max_out_bytes=1 << 20, host_pool_bytes=32 << 20,
                   device_arena=arena) as ctx:
        tasks = _submit_all(C, ctx, jobs)
        _check(C, tasks, jobs, want)
        base = arena.data_ptr()
        for t in tasks:
            assert base <= C.load().crystal_task_device_in(t.handle) < base + arena.numel()


def test_bound_input_from_registered_memory(C, oracle_mod):
    from paper_1005_1695_b300 import inputs

    n = 700_001
    src = C.page_aligned(3 * n)
    src[:] = inputs.uniform_unit(41, 0, 3 * n)
    C.host_register(src)
    try:
        with C.Context(max_in_bytes=1 << 20, max_out_bytes=1 << 20, device_pool_bytes=64 << 20,
                       host_pool_bytes=16 << 20) as ctx:
            h = ctypes.c_void_p()
            st = C.load().crystal_task_create_ex(ctx.handle, n, 16, 0, C.CRYSTAL_TASK_EXTERNAL_INPUT,
                                                ctypes.byref(h))
            assert st == C.CRYSTAL_OK
            t = C.Task(ctx, h.value, n, 16)
            ctx._tasks.add(t)
            assert C.load().crystal_task_host_in(t.handle) is None
            assert t.submit(DIRECT) == C.CRYSTAL_EINVAL  # nothing bound yet
            for k in range(3):
                view = src[k * n:(k + 1) * n]
                t.bind_input(view)
                assert t.submit(DIRECT) == C.CRYSTAL_OK
                assert t.wait(30 * SEC) == C.CRYSTAL_OK
                assert t.output()[:16] == oracle_mod.direct(view, 4096)
            assert C.load().crystal_task_bind_input(t.handle, None, 0) == C.CRYSTAL_EINVAL
            # a job with its own buffer can also be bound, and unbound again
            t2 = ctx.task_create(n, 16)
            t2.h_in[:] = src[:n]
            t2.bind_input(src[n:2 * n])
            assert t2.submit(DIRECT) == 0 and t2.wait(30 * SEC) == 0
            assert t2.output()[:16] == oracle_mod.direct(src[n:2 * n], 4096)
            t2.bind_input(None)
            assert t2.submit(DIRECT) == 0 and t2.wait(30 * SEC) == 0
            assert t2.output()[:16] == oracle_mod.direct(src[:n], 4096)
    finally:
        C.host_unregister(src)


def test_priority_jobs_overtake_queued_fifo_jobs(C):
    """Sequential mode: while a long job runs, five low-priority jobs and then one
    high-priority job are queued; the high one is dispatched next, the low
    ones after it in submission order."""
    with C.Context(max_in_bytes=64 << 20, max_out_bytes=8 << 20, device_pool_bytes=512 << 20,
                   host_pool_bytes=256 << 20, flags=C.CRYSTAL_FLAG_NO_OVERLAP) as ctx:
        n = 48 << 20
        big = ctx.task_create(n, C.sliding_out_bytes(n, 1 << 14))
        big.h_in[:] = 9
        low = [ctx.task_create(4096, 16) for _ in range(5)]
        high = ctx.task_create(4096, 16)
        for t in low + [high]:
            t.h_in[:] = 1
        assert high.set_priority(5) == 0
        assert big.submit(SLIDING) == 0
        import time

        deadline = time.time() + 5
        while big.timing()[1] == 0 and time.time() < deadline:  # wait until the long job is dispatched
            time.sleep(1e-5)
        assert big.timing()[1] > 0
        for t in low:
            assert t.submit(DIRECT) == 0
        assert high.submit(DIRECT) == 0
        for t in [big, high] + low:
            assert t.wait(60 * SEC) == 0
        d_high = high.timing()[1]
        d_low = [t.timing()[1] for t in low]
        assert big.timing()[1] < d_high < min(d_low)
        assert d_low == sorted(d_low)
        assert high.set_priority(0) == 0


def test_sha1_jobs_through_runtime(C, oracle_mod):
    from paper_1005_1695_b300 import inputs

    jobs = []
    for i in range(10):
        n = [65536, 300001, 0, 1 << 20, 77][i % 5]
        if i % 2:
            data = inputs.dedup_unit(29, i, n)
            jobs.append((C.CRYSTAL_KIND_SHA1_SLIDING, data, C.sliding_out_bytes(n, n // 256 + 16, 4),
                         C.params(mask=0x3FF, target=0x3FF)))
        else:
            data = inputs.uniform_unit(29, i, n)
            jobs.append((C.CRYSTAL_KIND_SHA1_DIRECT, data, 20, C.params(segment_bytes=2048)))
    want = _want(oracle_mod, jobs)
    with C.Context(max_in_bytes=2 << 20, max_out_bytes=1 << 20, device_pool_bytes=128 << 20,
                   host_pool_bytes=64 << 20, n_streams=3, flags=C.CRYSTAL_FLAG_GRAPHS, max_batch_jobs=4) as ctx:
        tasks = _submit_all(C, ctx, jobs)
        _check(C, tasks, jobs, want)


def test_wait_many_and_timing_many(C, oracle_mod):
    """One wait and one stamp read for a set of jobs: the first non-OK status
    in array order, a bounded wait that runs out, the argument checks, and no
    waiting from a callback."""
    L = C.load()
    from paper_1005_1695_b300 import inputs

    with C.Context(max_in_bytes=64 << 20, max_out_bytes=8 << 20, device_pool_bytes=512 << 20,
                   host_pool_bytes=256 << 20, n_streams=4, max_batch_jobs=4) as ctx:
        n = 300000
        small = C.sliding_out_bytes(n, 2)  # too few chunk records: EOVERFLOW
        outs = [C.sliding_out_bytes(n, n // 16), small, C.sliding_out_bytes(n, n // 16), 16]
        kinds = [SLIDING, SLIDING, SLIDING, DIRECT]
        tasks = []
        for i, (k, o) in enumerate(zip(kinds, outs)):
            t = ctx.task_create(n, o)
            t.h_in[:] = inputs.uniform_unit(31, i, n)
            tasks.append(t)
        p = C.params(mask=0x3F, target=0x3F)
        for t, k in zip(tasks, kinds):
            assert t.submit(k, p) == C.CRYSTAL_OK
        assert ctx.wait_many(tasks, 60 * SEC) == C.CRYSTAL_EOVERFLOW  # job 1, first non-OK in order
        assert [t.poll() for t in tasks] == [C.CRYSTAL_OK, C.CRYSTAL_EOVERFLOW, C.CRYSTAL_OK, C.CRYSTAL_OK]
        for i in (0, 2):
            st, want = oracle_mod.task(SLIDING, bytes(tasks[i].h_in), outs[i], mask=0x3F, target=0x3F)
            assert st == 0 and same_result(SLIDING, n, tasks[i].output(), want)
        stamps = ctx.timing_many(tasks)
        assert stamps.shape == (4, 3)
        for i, t in enumerate(tasks):
            assert tuple(int(x) for x in stamps[i]) == t.timing()
            assert 0 < stamps[i, 0] <= stamps[i, 1] <= stamps[i, 2]
        # all OK; the array can be built once and reused
        arr = ctx.task_array([tasks[0], tasks[2]])
        for _ in range(2):
            assert ctx.submit_many(arr, SLIDING, p) == C.CRYSTAL_OK
            assert ctx.wait_many(arr, 60 * SEC) == C.CRYSTAL_OK
        # a bounded wait that runs out, then completes
        big = ctx.task_create(48 << 20, C.sliding_out_bytes(48 << 20, 1 << 14))
        big.h_in[:] = 7
        assert big.submit(SLIDING) == C.CRYSTAL_OK
        assert ctx.wait_many([tasks[0], big], 0) == C.CRYSTAL_ETIMEDOUT
        assert ctx.wait_many([tasks[0], big], 60 * SEC) == C.CRYSTAL_OK
        # argument checks
        assert ctx.wait_many([], 0) == C.CRYSTAL_OK
        assert L.crystal_task_wait_many(None, 1, 0) == C.CRYSTAL_EINVAL
        never = ctx.task_create(100, 16)
        assert ctx.wait_many([tasks[0], never], 0) == C.CRYSTAL_EINVAL
        assert L.crystal_task_timing_many(None, 1, None) == C.CRYSTAL_EINVAL
        with C.Context(device_pool_bytes=16 << 20, host_pool_bytes=16 << 20) as other:
            o = other.task_create(100, 16)
            o.h_in[:] = 0
            assert o.submit(DIRECT) == C.CRYSTAL_OK and o.wait(10 * SEC) == C.CRYSTAL_OK
            assert ctx.wait_many([tasks[0], o], 0) == C.CRYSTAL_EINVAL  # two contexts
        # not from a completion callback
        seen = []
        handles = ctx.task_array([tasks[0]])

        @C.crystal_callback
        def cb(handle, status, user):
            seen.append(L.crystal_task_wait_many(handles, 1, 0))

        t = ctx.task_create(4096, 16)
        t.h_in[:] = 1
        assert t.submit(DIRECT, None, cb) == C.CRYSTAL_OK
        assert t.wait(30 * SEC) == C.CRYSTAL_OK
        assert seen == [C.CRYSTAL_EINVAL]


@pytest.mark.parametrize("flags", [0, 8], ids=["launches", "graphs"])
def test_bound_inputs_every_alignment_and_small_sizes(C, oracle_mod, flags):
    """Inputs read in place from registered memory at every offset mod 16, with
    sizes around 16-byte vectors and 16 KiB, and small outputs: the oracle's
    bytes, each bound input copied by its own DMA transfer."""
    from paper_1005_1695_b300 import inputs

    sizes = [1, 2, 15, 16, 17, 31, 33, 63, 64, 65, 100, 4095, 4096, 4097, 16383, 16384, 16385, 16400, 40000,
             300001]
    total = sum(s + 16 for s in sizes) * 2 + 4096
    src = C.page_aligned(total)
    src[:] = inputs.uniform_unit(77, 0, total)
    C.host_register(src)
    try:
        jobs = []
        pos = 0
        for i, n in enumerate(sizes * 2):
            off = pos + (i * 7) % 16
            kind = SLIDING if i % 4 == 3 else DIRECT
            osz = C.sliding_out_bytes(n, n // 64 + 8) if kind == SLIDING else 16
            p = C.params(mask=0x3F, target=0x3F) if kind == SLIDING else C.params(segment_bytes=1024)
            jobs.append((kind, off, n, osz, p))
            pos = off + n
        with C.Context(max_in_bytes=1 << 20, max_out_bytes=1 << 20, device_pool_bytes=256 << 20,
                       host_pool_bytes=64 << 20, n_streams=4, max_batch_jobs=8, flags=flags) as ctx:
            tasks = []
            for kind, off, n, osz, p in jobs:
                t = ctx.task_create(n, osz)
                t.bind_input(src[off:off + n])
                tasks.append(t)
            for t, (kind, off, n, osz, p) in zip(tasks, jobs):
                assert t.submit(kind, p) == C.CRYSTAL_OK
            assert ctx.wait_many(tasks, 60 * SEC) == C.CRYSTAL_OK
            for i, (t, (kind, off, n, osz, p)) in enumerate(zip(tasks, jobs)):
                st, w = oracle_mod.task(kind, src[off:off + n].tobytes(), osz, seg_bytes=p.segment_bytes,
                                        mask=p.mask, target=p.target)
                assert st == 0
                g = t.output()
                assert same_result(kind, n, g, w), f"job {i} n={n} off%16={off % 16}: " + \
                    first_difference(kind, n, g, w)
            st = ctx.stats()
            # bound inputs never merge; direct digests are written in place (no copy-out)
            n_sliding = sum(1 for j in jobs if j[0] == SLIDING)
            assert st.copies_dma >= len(jobs) and st.copies_dma <= len(jobs) + n_sliding
    finally:
        C.host_unregister(src)


@pytest.mark.parametrize("graphs", [0, 8], ids=["launches", "graphs"])
def test_launch_geometry_per_size_class_bit_exact(C, oracle_mod, graphs):
    """Every geometry choice (segment-kernel CTA size and CTAs per SM, window
    kernel CTAs per SM and register budget, chunk-segment CTAs per SM), set per
    batch size class, gives the oracle's bytes; bad fields are refused."""
    jobs = _jobs(C, count=30, seed=13)
    want = _want(oracle_mod, jobs)
    geoms = [C.geometry(seg_threads=64, seg_ctas_per_sm=1, win_ctas_per_sm=1, win_registers=64, digest_ctas_per_sm=1),
             C.geometry(seg_threads=256, seg_ctas_per_sm=2, win_ctas_per_sm=3, win_registers=32, digest_ctas_per_sm=2),
             C.geometry()]
    with C.Context(max_in_bytes=2 << 20, max_out_bytes=1 << 20, device_pool_bytes=256 << 20,
                   host_pool_bytes=128 << 20, n_streams=3, flags=graphs, max_batch_jobs=4) as ctx:
        for k in range(len(geoms)):
            for cls in range(C.CRYSTAL_SIZE_CLASSES):
                ctx.set_geometry(cls, geoms[(k + cls) % len(geoms)])
            g = ctx.get_geometry(1)
            assert g.seg_threads in (64, 128, 256) and g.win_registers in (32, 64) and g.seg_ctas_per_sm >= 1
            tasks = _submit_all(C, ctx, jobs)
            _check(C, tasks, jobs, want)
            for t in tasks:
                assert t.release() == C.CRYSTAL_OK
        got = ctx.get_geometry(2)  # the last round set class 2 to geoms[(2 + 2) % 3]
        assert (got.seg_threads, got.seg_ctas_per_sm, got.win_ctas_per_sm) == (256, 2, 3)
        L = C.load()
        for bad in (C.geometry(seg_threads=96), C.geometry(win_registers=48), C.geometry(reserved=1),
                    C.geometry(win_ctas_per_sm=65)):
            assert L.crystal_set_geometry(ctx.handle, 0, ctypes.byref(bad)) == C.CRYSTAL_EINVAL
        assert L.crystal_set_geometry(ctx.handle, 3, None) == C.CRYSTAL_EINVAL
        ctx.set_geometry(-1, None)
        assert ctx.get_geometry(2).seg_threads == 128


def test_adjacent_inputs_merge_into_one_copy_in_any_order(C, oracle_mod):
    """Jobs created one after another get adjacent pinned inputs at the same
    arena offsets as their device inputs; submitted in reverse order in one
    batch, their inputs still reach the GPU in one transfer (direct digests are
    written in place, so the batch has no copy back), and every digest is the
    oracle's."""
    from paper_1005_1695_b300 import inputs

    n, k = 65536 + 1000, 16
    with C.Context(max_in_bytes=1 << 20, max_out_bytes=1 << 10, device_pool_bytes=64 << 20,
                   host_pool_bytes=64 << 20, n_streams=1, max_batch_jobs=k, max_batch_bytes=64 << 20) as ctx:
        tasks = [ctx.task_create(n, 16) for _ in range(k)]
        data = [inputs.uniform_unit(21, i, n) for i in range(k)]
        for t, d in zip(tasks, data):
            t.h_in[:] = d
        before = ctx.stats().copies_dma
        assert ctx.submit_many(list(reversed(tasks)), DIRECT, C.params()) == C.CRYSTAL_OK
        assert ctx.wait_many(tasks, 30 * SEC) == C.CRYSTAL_OK
        s = ctx.stats()
        assert s.batches_launched == 1 and s.copies_dma - before == 1
        for t, d in zip(tasks, data):
            assert t.output()[:16] == oracle_mod.direct(d, 4096)


def test_alu_probe_kinds_work_and_arguments(C):
    """crystal_alu_probe: every kind launches and reports its work (windows
    for the two window kinds, instructions for the chains), the work grows
    with the iterations, and bad arguments are refused (EINVAL)."""
    import torch

    sink = torch.zeros(4, dtype=torch.uint8, device="cuda")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for kind in range(7):
        w1 = C.alu_probe(kind, 2, 1, sink)
        w4 = C.alu_probe(kind, 2, 4, sink)
        assert w1 > 0 and w4 == 4 * w1, kind
        if kind in (0, 1):  # eight windows per thread per iteration
            assert w1 == sms * 2 * 256 * 8
    torch.cuda.synchronize()
    L = C.load()
    s = torch.cuda.current_stream().cuda_stream
    assert L.crystal_alu_probe(7, 2, 1, 0, sink.data_ptr(), s, None) == C.CRYSTAL_EINVAL
    assert L.crystal_alu_probe(0, 0, 1, 0, sink.data_ptr(), s, None) == C.CRYSTAL_EINVAL
    assert L.crystal_alu_probe(0, 65, 1, 0, sink.data_ptr(), s, None) == C.CRYSTAL_EINVAL
    assert L.crystal_alu_probe(0, 2, 0, 0, sink.data_ptr(), s, None) == C.CRYSTAL_EINVAL
    assert L.crystal_alu_probe(0, 2, 1, 0, None, s, None) == C.CRYSTAL_EINVAL


def test_get_config_reports_the_context(C):
    with C.Context(max_in_bytes=3 << 20, max_out_bytes=5 << 10, device_pool_bytes=48 << 20,
                   host_pool_bytes=40 << 20, n_streams=3, max_batch_jobs=12, flags=C.CRYSTAL_FLAG_GRAPHS) as ctx:
        cfg = ctx.config()
        assert (cfg.max_in_bytes, cfg.max_out_bytes) == (3 << 20, 5 << 10)
        assert (cfg.device_pool_bytes, cfg.host_pool_bytes) == (48 << 20, 40 << 20)
        assert cfg.n_streams == 3 and cfg.max_batch_jobs == 12 and cfg.flags == C.CRYSTAL_FLAG_GRAPHS
    with C.Context(max_in_bytes=1 << 20, max_out_bytes=1 << 10, device_pool_bytes=16 << 20,
                   host_pool_bytes=16 << 20, n_streams=4, max_batch_jobs=12,
                   flags=C.CRYSTAL_FLAG_NO_BATCH) as ctx:
        assert ctx.config().max_batch_jobs == 1  # one job per launch


def test_direct_job_moves_the_bytes(C):
    """crystal_direct_job (the overhead experiment's baseline): copy in, an
    empty kernel, copy out.  With the output read back from the input's
    device buffer, the bytes come back unchanged."""
    import torch

    n = 300_001
    h_in = torch.randint(0, 256, (n,), dtype=torch.uint8).pin_memory()
    h_out = torch.zeros(n, dtype=torch.uint8).pin_memory()
    d = torch.empty(n, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    L = C.load()
    assert L.crystal_direct_job(h_in.data_ptr(), d.data_ptr(), n, h_out.data_ptr(), d.data_ptr(), n,
                                s.cuda_stream) == C.CRYSTAL_OK
    assert torch.equal(h_in, h_out)
