"""Job-stream drivers over the C-ABI job runtime.

These run a stream of data units through ``crystal_task_*`` the way an
application of the paper's framework does (Section 2.2: a steady stream of
data units, one job each; Section 5.2: a stream of jobs hashed by StoreGPU),
in the forms the paper compares (Section 5.2, Figure 7):

* ``pooled``          buffers from the pool allocated at init, several
                      streams, outstanding jobs batched per launch; the data
                      are produced straight into the jobs' pinned buffers
                      (Section 2.1's advice) before the stream starts.
* ``pooled_staged``   the same runtime fed from pageable memory: the
                      library's staging ring (``crystal_stream_staged``) of
                      ``depth`` pooled jobs, refilled by ``copy_threads`` C++
                      threads (one host copy per unit inside the timed region).
* ``no_overlap``      pooled buffers, one stream, one job at a time: copy-in,
                      kernel and copy-out of a job never overlap another job.
* ``per_job_malloc``  every job allocates its pinned and device buffers when
                      it is created and frees them when released (the
                      allocation the pool removes), data staged from pageable
                      memory; ``depth`` jobs in flight.
* ``plain``           ``per_job_malloc`` with one stream and one job at a time:
                      allocate, copy in, hash, copy out, free — job by job.

All hashing runs in ``libcrystal.so``; this module only creates, fills,
submits and waits on jobs and records host clock stamps.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np

from . import crystal as C

MODES = ("pooled", "pooled_staged", "no_overlap", "per_job_malloc", "plain")

_FLAGS = {
    "pooled": 0,
    "pooled_staged": 0,
    "no_overlap": C.CRYSTAL_FLAG_NO_OVERLAP | C.CRYSTAL_FLAG_NO_BATCH,
    "per_job_malloc": C.CRYSTAL_FLAG_NO_POOL,
    "plain": C.CRYSTAL_FLAG_NO_POOL | C.CRYSTAL_FLAG_NO_OVERLAP | C.CRYSTAL_FLAG_NO_BATCH,
}


@dataclass
class StreamResult:
    mode: str
    units: int
    bytes: int
    seconds: float
    latencies_ms: List[float]
    outputs: Dict[int, bytes] = field(default_factory=dict)
    statuses: List[int] = field(default_factory=list)

    @property
    def gbs(self) -> float:
        return self.bytes / self.seconds / 1e9

    def latency(self, q: float) -> float:
        return float(np.percentile(self.latencies_ms, q)) if self.latencies_ms else 0.0


def _used(kind: int, n: int, out: np.ndarray) -> int:
    if kind in C.DIRECT_KINDS:
        return C.digest_size(kind)
    words = (n + 31) // 32
    n_chunks = int(out[0:4].view(np.uint32)[0])
    flags = int(out[4:8].view(np.uint32)[0])
    return 8 + 4 * words + (0 if flags & 1 else (4 + C.digest_size(kind)) * n_chunks)


def run_stream(mode: str, unit: Callable[[int], np.ndarray], n_units: int, unit_bytes: int, kind: int,
               p: C.crystal_hash_params, out_size: int, *, streams: int = 8, batch_jobs: int = 8,
               depth: int = 24, graphs: bool = True, device: int = 0, keep: Sequence[int] = (),
               device_pool_bytes: Optional[int] = None, host_pool_bytes: Optional[int] = None,
               copy_threads: int = 8, warm: bool = True) -> StreamResult:
    """Hash ``n_units`` units (``unit(i)`` returns unit i's bytes) in ``mode``.

    Returns wall time of the stream (first submit to last completion seen by
    the application), per-job latencies (submit to completion, master-thread
    stamps) and the used output bytes of the units listed in ``keep``.  With
    ``warm`` the context's batch graphs are captured before the stream
    (crystal_prepare_graphs), a set-up step like the pools, and the resident
    forms run the jobs once untimed.  Either way the timed pass hashes inputs
    the application has just written into the jobs' pinned buffers (a pass
    over 16 GiB of pinned inputs the DMA engines had already read, not
    written again, was measured 5% slower on the host link: 51.6 against
    54.5 GB/s)."""
    if mode not in MODES:
        raise ValueError(mode)
    flags = _FLAGS[mode] | (C.CRYSTAL_FLAG_GRAPHS if graphs and mode in ("pooled", "pooled_staged") else 0)
    keep = set(keep)
    scratch = C.scratch_bytes(kind, unit_bytes, out_size, p)
    per_job_dev = unit_bytes + out_size + scratch + 3 * 256
    resident = mode in ("pooled", "no_overlap")
    ring = n_units if resident else (1 if mode == "plain" else min(depth, n_units))
    dev_pool = device_pool_bytes or (ring * per_job_dev + (64 << 20))
    host_pool = host_pool_bytes or (ring * (unit_bytes + out_size + 512) + (16 << 20))
    ctx = C.Context(max_in_bytes=unit_bytes, max_out_bytes=out_size, device_pool_bytes=dev_pool,
                    host_pool_bytes=host_pool, n_streams=streams, device=device, flags=flags,
                    max_batch_jobs=batch_jobs, max_batch_bytes=batch_jobs * max(unit_bytes, 1))
    res = StreamResult(mode, n_units, n_units * unit_bytes, 0.0, [])
    try:
        if warm:
            ctx.prepare_graphs()  # a set-up step of the context (nothing without graphs)
        if mode == "pooled_staged":
            src = [unit(i) for i in range(n_units)]  # pageable application memory
            st, rr, wall, outs = ctx.stream_staged(src, kind, out_size, p, copy_threads=copy_threads,
                                                   ring_jobs=ring, keep_outputs=bool(keep))
            res.seconds = wall / 1e9
            res.statuses = [int(x) for x in rr["status"]]
            res.latencies_ms = ((rr["done_ns"].astype(np.float64) - rr["submit_ns"].astype(np.float64)) / 1e6).tolist()
            for i in keep:
                res.outputs[i] = outs[i, :int(rr["used_bytes"][i])].tobytes()
        elif resident:
            tasks = [ctx.task_create(unit_bytes, out_size) for _ in range(n_units)]
            handles = ctx.task_array(tasks)
            if warm:
                # one untimed pass (the slots' streams, events and mapped
                # descriptor pages used once), then fresh inputs as below
                for i, t in enumerate(tasks):
                    t.h_in[:] = unit(i)
                C.check(ctx.submit_many(handles, kind, p), "crystal_task_submit_many")
                ctx.wait_many(handles, 600_000_000_000)
            for i, t in enumerate(tasks):
                t.h_in[:] = unit(i)  # produced into the job's pinned buffer, before the stream
            t0 = time.perf_counter()
            C.check(ctx.submit_many(handles, kind, p), "crystal_task_submit_many")
            ctx.wait_many(handles, 600_000_000_000)
            res.seconds = time.perf_counter() - t0
            stamps = ctx.timing_many(handles)
            for i, t in enumerate(tasks):
                res.statuses.append(t.poll())
                res.latencies_ms.append(float(stamps[i, 2] - stamps[i, 0]) / 1e6)
                if i in keep:
                    res.outputs[i] = t.h_out[:_used(kind, unit_bytes, t.h_out)].tobytes()
                t.release()
        else:
            # per-job allocation: each job allocated, filled from pageable
            # application memory, submitted, waited for and freed
            src = [unit(i) for i in range(n_units)]
            inflight = []  # (unit index, task)

            def retire():
                i, t = inflight.pop(0)
                res.statuses.append(t.wait(600_000_000_000))
                s, _, d = t.timing()
                res.latencies_ms.append((d - s) / 1e6)
                if i in keep:
                    res.outputs[i] = t.h_out[:_used(kind, unit_bytes, t.h_out)].tobytes()
                t.release()

            t0 = time.perf_counter()
            for i in range(n_units):
                if len(inflight) >= ring:
                    retire()
                t = ctx.task_create(unit_bytes, out_size)
                t.h_in[:] = src[i]
                C.check(t.submit(kind, p), "crystal_task_submit")
                inflight.append((i, t))
            while inflight:
                retire()
            res.seconds = time.perf_counter() - t0
    finally:
        ctx.shutdown()
    return res


# ---- served stream --------------------------------------------------------------

def make_trace(seed: int, n: int, rate_per_s: float, source_bytes: int, *, median: int = 256 << 10,
               sigma: float = 1.5, cap: int = 64 << 20, p_sliding: float = 0.3, window: int = 20,
               capture_every: int = 0, chunk_room: int = 4):
    """An open-loop request trace: Poisson arrivals at ``rate_per_s``,
    lognormal sizes (median, sigma, capped), a ``p_sliding`` share of
    sliding-window requests, each request a window of the source arena at a
    seeded offset.  Sliding outputs have room for ``chunk_room`` times the
    expected chunk count (one chunk per 8 KiB) plus 64.  Every
    ``capture_every``-th request (0: none) has its output captured; returns
    (requests, capture_bytes)."""
    from . import inputs

    sizes = inputs.lognormal_sizes(seed, n, median=median, sigma=sigma, cap=min(cap, source_bytes))
    arrivals = inputs.poisson_arrivals(seed, n, rate_per_s)
    sliding = inputs.kind_mix(seed, n, p_sliding)
    offs = inputs.rng(seed, inputs.TAG_SIZES, 7).integers(0, 1 << 62, size=n) % (source_bytes - sizes + 1)
    req = np.zeros(n, dtype=C.REQUEST_DTYPE)
    req["arrival_ns"] = np.round(arrivals * 1e9).astype(np.uint64)
    req["src_offset"] = offs
    req["size"] = sizes
    req["kind"] = np.where(sliding, C.CRYSTAL_KIND_MD5_SLIDING, C.CRYSTAL_KIND_MD5_DIRECT)
    set_out_sizes(req, chunk_room)
    cap_bytes = assign_capture(req, capture_every)
    return req, cap_bytes


def set_out_sizes(req, chunk_room: int = 4) -> None:
    """Output bytes of every request from its kind and size: the digest for
    direct requests; for sliding ones the header, the bitmap and room for
    ``chunk_room`` times the expected chunk count (one chunk per 8 KiB on
    random data) plus 64 records."""
    out = np.empty(len(req), dtype=np.uint64)
    for i in range(len(req)):
        k, n = int(req["kind"][i]), int(req["size"][i])
        out[i] = C.sliding_out_bytes(n, chunk_room * (n // 8192) + 64, k) if k in C.SLIDING_KINDS else \
            C.digest_size(k)
    req["out_size"] = out


def assign_capture(req, every: int = 1) -> int:
    """Give every ``every``-th request (0: none) a 16-byte aligned slot of its
    ``out_size`` bytes in one capture buffer; returns the buffer's size."""
    req["capture_offset"] = C.NO_CAPTURE
    cap_bytes = 0
    if every:
        for i in range(0, len(req), every):
            req["capture_offset"][i] = cap_bytes
            cap_bytes += int(req["out_size"][i] + 15) // 16 * 16
    return cap_bytes


def serve_trace(req, source, *, device_pool_bytes: int, host_pool_bytes: int, streams: int = 8,
                batch_jobs: int = 8, copy_threads: int = 4, device: int = 0, capture_bytes: int = 0,
                graphs: bool = True, direct=None, sliding=None, source_pinned: bool = False,
                arrival_order: bool = False, bypass_ns: int = 0, ring_bytes: int = 0,
                ring_max_request: int = 0):
    """Run a trace through crystal_serve on a fresh context sized to the pools.
    With ``source_pinned`` the source is page-locked for the run and jobs read
    their input from it directly; ``arrival_order`` / ``bypass_ns`` set the
    admission policy; ``ring_bytes`` / ``ring_max_request`` stage small
    requests through an input ring.  Returns (status, results, wall_ns,
    capture)."""
    max_in = int(req["size"].max()) if len(req) else 1
    max_out = int(req["out_size"].max()) if len(req) else 16
    ctx = C.Context(max_in_bytes=max(max_in, 1), max_out_bytes=max(max_out, 16),
                    device_pool_bytes=device_pool_bytes, host_pool_bytes=host_pool_bytes, n_streams=streams,
                    device=device, max_batch_jobs=batch_jobs, max_batch_bytes=max(batch_jobs << 20, 32 << 20),
                    flags=C.CRYSTAL_FLAG_GRAPHS if graphs else 0)
    capture = np.zeros(max(capture_bytes, 16), dtype=np.uint8) if capture_bytes else None
    ctx.prepare_graphs()
    if source_pinned:
        C.host_register(source)
    try:
        st, res, wall = ctx.serve(source, req, direct=direct, sliding=sliding, capture=capture,
                                  copy_threads=copy_threads, source_pinned=source_pinned,
                                  arrival_order=arrival_order, bypass_ns=bypass_ns, ring_bytes=ring_bytes,
                                  ring_max_request=ring_max_request)
    finally:
        ctx.shutdown()
        if source_pinned:
            C.host_unregister(source)
    return st, res, wall, capture


def latency_ms(req, res) -> np.ndarray:
    """Request latency: completion minus arrival (admission wait included)."""
    return (res["done_ns"].astype(np.float64) - req["arrival_ns"].astype(np.float64)) / 1e6


def make_batch(seed: int, n: int, source_bytes: int, *, lo: int = 4096, hi: int = 16 << 20,
               p_sliding: float = 0.2, chunk_room: int = 4, capture: bool = False):
    """``n`` units of log-uniform size in [lo, hi], a ``p_sliding`` share of
    them sliding-window, all available at once (arrival 0), each a window of
    the source arena at a seeded offset.  Returns (requests, capture_bytes)."""
    from . import inputs

    sizes = inputs.loguniform_sizes(seed, n, lo=lo, hi=min(hi, source_bytes))
    sliding = inputs.kind_mix(seed, n, p_sliding)
    offs = inputs.rng(seed, inputs.TAG_SIZES, 9).integers(0, 1 << 62, size=n) % (source_bytes - sizes + 1)
    req = np.zeros(n, dtype=C.REQUEST_DTYPE)
    req["src_offset"] = offs
    req["size"] = sizes
    req["kind"] = np.where(sliding, C.CRYSTAL_KIND_MD5_SLIDING, C.CRYSTAL_KIND_MD5_DIRECT)
    set_out_sizes(req, chunk_room)
    cap_bytes = assign_capture(req, 1 if capture else 0)
    return req, cap_bytes
