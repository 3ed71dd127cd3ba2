"""Benchmark of the hashing hot path on B300.

Default workload (one step): 256 units of 1 MiB, half of each unit repeated
8 KiB blocks from a seeded pool of 64, MD5 sliding-window hashing with a
20-byte window at every byte offset, boundary where
(first digest word & 0x1FFF) == 0x1FFF, then a direct hash (4 KiB segments)
of every resulting chunk.  That step runs every stage of the path: window
MD5s and bitmap, chunk extraction, chunk segment MD5s, digest of digests,
and (end to end) the pooled pinned buffers, copy-in, copy-out and the
master thread's batching, polling and completion.

* ``value``  -- hashed GB/s with the inputs already resident in HBM: the
  kernel chain launched through the C ABI on a device-resident batch.
* ``e2e``    -- the same metric through the job API with pinned host buffers:
  submit, copy-in, kernels, copy-out and completion inside the timed region.
* ``roofline`` -- the window kernel (the dominant one) against the integer
  issue rate of the GPU.
* ``cpu_baseline`` -- the CPU oracle on the host cores, on a bounded sample.

``--impl reference`` times the CPU oracle as the reference arm on the same
workload (bounded sample per step).  Under torchrun every rank runs its own
replica (units are independent; there is no exchange step).

Other workloads (``--workload``) print their own lines for the design
notes; the default one is the headline.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "end-to-end hashed GB/s (host→digests) and fraction of host-link roofline; p50/p99 latency"
GB = 1e9

# Algorithmic integer operations of one window (w = 20, one MD5 block, only
# the first digest word is needed): 61 of the 64 steps (A is final after
# step 61); a step is one 3-input logic op, one 3-input add (two when its
# message word is data rather than a padding constant), one rotate, one
# add; 19 of the 61 steps use one of the 5 data words.  Then the
# feed-forward add, the mask and the compare.
OPS_PER_WINDOW_W20 = 61 * 4 + 19 + 3
# SHA-1 window (w = 20, one block, the first digest word needs all 80 steps):
# per step a rotate of a, the 3-input round function, two 3-input adds (a<<<5,
# f, e, constant, schedule word) and the rotate of b; from step 16 on the
# schedule word costs two 3-input XORs and a rotate; then the feed-forward
# add, the mask and the compare.
OPS_PER_WINDOW_SHA1_W20 = 80 * 5 + 64 * 3 + 3
SM_COUNT_B300 = 148
INT_LANES_PER_SM = 128  # 4 schedulers x one 32-lane instruction per clock

# DRAM bytes (read + write) of the window kernel per 1 MiB sliding unit, from one
# ncu capture of 160 units (traffic grows with the units processed), valid only
# for the kernel sources it was taken on (checked by hash; otherwise null).
WINDOW_TRAFFIC_PER_UNIT = (168.128512e6 + 14.240768e6) / 160
WINDOW_TRAFFIC_SOURCES = "36822ebde71ff91b"


def _kernel_sources_hash() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in ("kernels.cu", "md5_device.cuh"):
        with open(os.path.join(ROOT, "paper_1005_1695_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _mean_ci(xs) -> dict:
    """Mean and 95% confidence half-width (normal approximation) of per-step
    times, with their spread: the paper's reporting (means over repeated runs
    with 95% intervals, Section 5)."""
    a = np.asarray(xs, dtype=np.float64)
    half = 1.96 * float(a.std(ddof=1)) / float(np.sqrt(len(a))) if len(a) > 1 else 0.0
    return {"mean": round(float(a.mean()), 4), "ci95": round(half, 4), "min": round(float(a.min()), 4),
            "max": round(float(a.max()), 4), "n": int(len(a))}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seed(seed: int, rank: int) -> int:
    """Each replica hashes its own synthetic data (weak scaling)."""
    return seed + rank


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """Largest value of x over the ranks (the slowest replica sets the time)."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_gbs(ws: int, bytes_per_rank: int, steps: int, seconds: float) -> float:
    """Whole-job throughput: every rank's bytes over the slowest rank's time."""
    return ws * bytes_per_rank * steps / seconds / GB


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1].split()[0]))
                smax.append(float(parts[2].split()[0]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measure_link(torch, dev, total: int, n_streams: int = 8, chunk: int = 8 << 20, reps: int = 3,
                 out_fraction: float = 0.0) -> dict:
    """Pinned host <-> device copy bandwidth: one stream copying ``total`` bytes
    at once, ``n_streams`` streams copying ``chunk``-byte pieces concurrently
    (which can use several copy engines), and -- when ``out_fraction`` > 0 --
    ``total`` bytes in while ``out_fraction`` x ``total`` bytes come back on a
    second stream (both directions share the link).  Best of ``reps``.

    The pinned buffer is allocated pinned and written by one thread: filling
    it with a multi-threaded torch copy leaves torch's worker threads spinning
    on every core for a while, and host-to-device copies measured meanwhile
    were up to 30% slower on B300 hosts with 16 cores."""
    pinned = torch.empty(total, dtype=torch.uint8, pin_memory=True)
    pinned.numpy()[:] = 1
    dbuf = torch.empty(total, dtype=torch.uint8, device=dev)
    streams = [torch.cuda.Stream(device=dev) for _ in range(n_streams)]
    n_out = int(total * out_fraction) & ~4095
    if n_out:
        pinned_out = torch.empty(n_out, dtype=torch.uint8, pin_memory=True)
        dout = torch.ones(n_out, dtype=torch.uint8, device=dev)

    def timed(h2d: bool, multi: bool, duplex: bool = False) -> float:
        best = 0.0
        for _ in range(reps + 1):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            cur = torch.cuda.current_stream()
            a.record(cur)
            if duplex:
                for s in streams[:2]:
                    s.wait_event(a)
                with torch.cuda.stream(streams[0]):
                    dbuf.copy_(pinned, non_blocking=True)
                with torch.cuda.stream(streams[1]):
                    pinned_out.copy_(dout, non_blocking=True)
                for s in streams[:2]:
                    cur.wait_stream(s)
            elif not multi:
                (dbuf.copy_(pinned, non_blocking=True) if h2d else pinned.copy_(dbuf, non_blocking=True))
            else:
                for s in streams:
                    s.wait_event(a)
                for i, off in enumerate(range(0, total, chunk)):
                    with torch.cuda.stream(streams[i % n_streams]):
                        d, h = dbuf[off:off + chunk], pinned[off:off + chunk]
                        (d.copy_(h, non_blocking=True) if h2d else h.copy_(d, non_blocking=True))
                for s in streams:
                    cur.wait_stream(s)
            b.record(cur)
            torch.cuda.synchronize()
            moved = total + (n_out if duplex else 0)
            best = max(best, moved / (a.elapsed_time(b) / 1e3) / GB)
        return best

    out = {"h2d_single_gbs": timed(True, False), "h2d_multi_gbs": timed(True, True),
           "d2h_single_gbs": timed(False, False), "d2h_multi_gbs": timed(False, True)}
    if n_out:
        out["duplex_gbs"] = timed(True, False, duplex=True)
    out = {k: round(v, 2) for k, v in out.items()}
    out["how"] = (f"torch pinned copies of {total >> 20} MiB: one stream, and {n_streams} streams x {chunk >> 20} MiB"
                  + (f"; duplex: {total >> 20} MiB in while {n_out >> 20} MiB come back, bytes of both per second"
                     if n_out else ""))
    del pinned, dbuf
    return out


def measure_int_pipes(torch, dev, C, ctas_per_sm: int = 16) -> dict:
    """The integer-pipe microbenchmarks of the library (crystal_alu_probe), on
    register data only, each timed with CUDA events on its stream (best of 5
    after a warm-up launch): the 20-byte window hash of MD5 and of SHA-1 as the
    window kernel computes it (windows/s), and single-instruction chains on
    one pipe (LOP3, funnel shift, three-input add, IMAD) or two (LOP3 and IMAD
    alternately: the dual-issue rate), in instructions/s.  Every launch runs
    for milliseconds (the chains 2,000 iterations), so that launch latency and
    the clock's ramp do not lower a peak."""
    sink = torch.zeros(4, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    iters = {"md5_windows": 400, "sha1_windows": 150}
    out = {}
    for name, kind in C.PROBE_KINDS.items():
        it = iters.get(name, 2000)
        with torch.cuda.stream(stream):
            C.alu_probe(kind, ctas_per_sm, max(1, it // 10), sink, stream)
            best = None
            for _ in range(5):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                work = C.alu_probe(kind, ctas_per_sm, it, sink, stream)
                b.record(stream)
                b.synchronize()
                ms = a.elapsed_time(b)
                best = ms if best is None else min(best, ms)
        out[name] = work / (best / 1e3)
    return out


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ---- workload ---------------------------------------------------------------------

def sliding_workload(seed: int, units: int, unit_bytes: int) -> np.ndarray:
    from paper_1005_1695_b300 import inputs

    pool = inputs.dedup_pool(seed)
    host = np.empty(units * unit_bytes, dtype=np.uint8)
    for u in range(units):
        inputs.dedup_unit(seed, u, unit_bytes, pool=pool, out=host[u * unit_bytes:(u + 1) * unit_bytes])
    return host


def cpu_oracle_rate(host: np.ndarray, unit_bytes: int, units: int, cores: int, params: dict, kind: int = 2,
                    results: dict = None) -> dict:
    """The oracle (as it stands) on ``units`` units over ``cores`` host threads.
    With ``results`` (unit -> the GPU's used output bytes for that unit), the
    oracle's output of each of those units is compared with them: the line's
    ``verified`` record."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor

    oracle.build()
    out_size = 8 + 4 * ((unit_bytes + 31) // 32) + (4 + oracle.digest_bytes(kind)) * 1024

    def one(u):
        return oracle.task(kind, host[u * unit_bytes:(u + 1) * unit_bytes], out_size, **params)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        outs = list(ex.map(one, range(units)))
    dt = time.perf_counter() - t0
    assert all(st == 0 for st, _ in outs)
    line = {"value": units * unit_bytes / dt / GB, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"{units} of the workload's 1 MiB units (sliding window w=20 + chunk direct hash), "
                      f"{cores} threads, {dt:.1f} s"}
    if results is not None:
        checked = [u for u in sorted(results) if u < units]
        bad = [u for u in checked if outs[u][1][:len(results[u])] != results[u]]
        line["_verified"] = {"units_checked": len(checked), "bit_exact": len(checked) - len(bad),
                             "mismatched_units": bad[:8], "against": "the oracle, every output byte"}
    return line


def cpu_oracle_detail(host: np.ndarray, unit_bytes: int, cores: int, params: dict) -> dict:
    """The oracle's rates on one host core and on all of them: plain MD5, direct
    hashing (4 KiB segments) and the sliding-window job, each on a few units of
    the workload (a few seconds of CPU in all)."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor

    oracle.build()
    units = [host[u * unit_bytes:(u + 1) * unit_bytes] for u in range(min(len(host) // unit_bytes, cores))]
    out_size = 8 + 4 * ((unit_bytes + 31) // 32) + 20 * 1024

    def rate(fn, items, threads):
        t0 = time.perf_counter()
        if threads == 1:
            for x in items:
                fn(x)
        else:
            with ThreadPoolExecutor(max_workers=threads) as ex:
                list(ex.map(fn, items))
        return round(len(items) * unit_bytes / (time.perf_counter() - t0) / GB, 4)

    md5 = oracle.md5
    direct = lambda x: oracle.direct(x, 4096)
    sliding = lambda x: oracle.task(2, x, out_size, **params)
    return {"unit": "GB/s", "cores": cores, "kind": "oracle",
            "md5_1core": rate(md5, units * 4, 1), "md5_all_cores": rate(md5, units * 4, cores),
            "direct_1core": rate(direct, units * 4, 1), "direct_all_cores": rate(direct, units * 4, cores),
            "sliding_1core": rate(sliding, units[:1], 1), "sliding_all_cores": rate(sliding, units, cores),
            "sample": f"{len(units)} of the workload's {unit_bytes >> 20} MiB units (x4 for MD5 and direct)"}


# ---- our arm ------------------------------------------------------------------------

def run_ours(args, ws, rank, local):
    import torch

    from paper_1005_1695_b300 import crystal as C

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    C.load()
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    def slowest(x: float) -> float:
        return max_over_ranks(x, dist, dev)

    U, N = args.units, args.unit_bytes
    p = C.params(window_bytes=20, mask=0x1FFF, target=0x1FFF, chunk_segment_bytes=4096)
    KIND = C.CRYSTAL_KIND_SHA1_SLIDING if args.hash == "sha1" else C.CRYSTAL_KIND_MD5_SLIDING
    gpu_results = {}  # unit -> used output bytes from the job API
    ops_per_window = OPS_PER_WINDOW_SHA1_W20 if args.hash == "sha1" else OPS_PER_WINDOW_W20
    out_size = C.sliding_out_bytes(N, args.max_chunks, KIND)
    host = sliding_workload(rank_seed(args.seed, rank), U, N)
    total_bytes = U * N

    # ---- value: inputs resident in HBM, kernel chain through the C ABI ----
    d_in = torch.from_numpy(host).to(dev)
    batch = C.DeviceBatch(d_in, [u * N for u in range(U)], [N] * U, [KIND] * U, p, out_sizes=[out_size] * U)
    desc_host = torch.from_numpy(batch.host_desc).pin_memory()
    torch.cuda.synchronize()
    stream = torch.cuda.Stream(device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    ev_step = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]

    def step(i=None):
        with torch.cuda.stream(stream):
            if i is not None:
                ev_step[i][0].record(stream)
            batch.d_desc.copy_(desc_host, non_blocking=True)
            if i is not None:
                ev[i][0].record(stream)
            batch.launch_sliding_windows(stream)
            if i is not None:
                ev[i][1].record(stream)
            batch.launch_sliding_chunks(stream)
            batch.launch_sliding_digests(stream)
            if i is not None:
                ev_step[i][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    launches0 = C.kernel_launches()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(i)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t0
    launches_value = C.kernel_launches() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev_step]
    win_ms = [a.elapsed_time(b) for a, b in ev]
    dev_ms = slowest(float(np.sum(step_ms)))
    value = aggregate_gbs(ws, total_bytes, args.steps, dev_ms / 1e3)
    assert batch.device_status() == 0

    # ---- e2e: job API, pinned host buffers, copies inside the timed region ----
    if "e2e" in args.legs:
        n_sets = max(1, args.e2e_sets)
        pool_dev = int(n_sets * (total_bytes + U * (out_size + C.scratch_bytes(KIND, N, out_size, p) + 4096))
                       + (64 << 20))
        pool_host = int(n_sets * (total_bytes + U * (out_size + 4096)) + (16 << 20))
        ctx = C.Context(max_in_bytes=N, max_out_bytes=out_size, device_pool_bytes=pool_dev,
                        host_pool_bytes=pool_host, n_streams=args.streams, max_batch_jobs=args.batch_jobs,
                        max_batch_bytes=args.batch_jobs * N, device=local,
                        flags=C.CRYSTAL_FLAG_GRAPHS if args.graphs else 0)
        # n_sets job sets of U units each (the same bytes), used in turn: step
        # k + 1 is submitted before step k is waited for, as a streaming
        # application keeps the pipeline full
        sets = []
        for _ in range(n_sets):
            tasks = [ctx.task_create(N, out_size) for _ in range(U)]
            for u, t in enumerate(tasks):
                t.h_in[:] = host[u * N:(u + 1) * N]
            sets.append((tasks, ctx.task_array(tasks)))

        def run_steps(n_steps, kind):
            """n_steps steps, each one submit of a job set and one wait for it
            (one call each), n_sets - 1 steps ahead; returns the stamps."""
            stamps = []
            for k in range(min(n_sets - 1, n_steps)):
                C.check(ctx.submit_many(sets[k % n_sets][1], kind, p), "submit_many")
            for i in range(n_steps):
                if i + n_sets - 1 < n_steps:
                    C.check(ctx.submit_many(sets[(i + n_sets - 1) % n_sets][1], kind, p), "submit_many")
                h = sets[i % n_sets][1]
                C.check(ctx.wait_many(h, 60_000_000_000), "wait_many")
                stamps.append(ctx.timing_many(h))
            return stamps

        run_steps(max(args.warmup, n_sets), KIND)
        # the job outputs must equal the device-resident outputs, unit by unit
        got_dev = batch.outputs()
        for tasks, _ in sets:
            for u in range(0, U, max(1, U // 16)):
                n_chunks = int.from_bytes(got_dev[u][:4], "little")
                used = 8 + 4 * (N // 32) + (4 + C.digest_size(KIND)) * n_chunks
                assert tasks[u].output()[:used] == got_dev[u][:used], "job output differs from device batch output"
        lat = []
        launches1 = C.kernel_launches()
        barrier()
        t0 = time.perf_counter()
        stamps = run_steps(args.steps, KIND)
        barrier()
        e2e_wall = slowest(time.perf_counter() - t0)
        for tm in stamps:
            lat.extend(((tm[:, 2] - tm[:, 0]).astype(np.float64) / 1e6).tolist())
        # time between consecutive steps' last completions (steps overlap, so
        # this spacing, not a step's own span, is its share of the wall time)
        done = np.array([float(tm[:, 2].max()) for tm in stamps]) / 1e6
        e2e_step_ms = np.diff(done).tolist()
        launches = launches_value + C.kernel_launches() - launches1
        e2e_value = aggregate_gbs(ws, total_bytes, args.steps, e2e_wall)
        # results of the units the CPU baseline leg will also hash (checked there)
        tasks0 = sets[0][0]
        for u in range(min(U, args.check_units)):
            o = tasks0[u].output()
            gpu_results[u] = o[:8 + 4 * ((N + 31) // 32) + (4 + C.digest_size(KIND)) * int.from_bytes(o[:4], "little")]
        # the same job shapes with the dummy kernel (copies only): the transfer ceiling
        t1 = time.perf_counter()
        run_steps(args.steps, C.CRYSTAL_KIND_NOP)
        copy_only = aggregate_gbs(ws, total_bytes, args.steps, slowest(time.perf_counter() - t1))
    else:
        e2e_value, lat, e2e_wall, launches, copy_only = None, [0.0], None, launches_value, None
        tasks, ctx = [], None
    # integer-pipe microbenchmarks, inside the clock record of the timed legs
    pipes = measure_int_pipes(torch, dev, C)
    clock_info = clocks.stop()

    # ---- host link (pinned copies) measured on this GPU ----
    out_bytes = U * out_size
    link = measure_link(torch, dev, total_bytes, out_fraction=out_bytes / total_bytes)
    h2d = max(link["h2d_single_gbs"], link["h2d_multi_gbs"])
    d2h = max(link["d2h_single_gbs"], link["d2h_multi_gbs"])
    # both directions at once share the link: input rate when the outputs
    # come back concurrently
    duplex_in = link["duplex_gbs"] * total_bytes / (total_bytes + out_bytes)

    # ---- roofline of the window kernel ----
    windows = U * (N - 20 + 1)
    win_avg_s = float(np.mean(win_ms)) / 1e3
    achieved = windows * ops_per_window / win_avg_s / 1e12
    peaks = _peaks()
    traffic = None
    if _kernel_sources_hash() == WINDOW_TRAFFIC_SOURCES and N == 1 << 20 and args.hash == "md5":
        traffic = round(WINDOW_TRAFFIC_PER_UNIT * U)
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    nominal = SM_COUNT_B300 * INT_LANES_PER_SM * sm_max * 1e6 / 1e12
    peak = pipes["lop3_imad"] / 1e12  # measured: the most int32 instructions the SMs issue per second
    mix_name = "sha1_windows" if args.hash == "sha1" else "md5_windows"
    mix_ceiling = pipes[mix_name] * ops_per_window / 1e12  # the window hash itself, no memory
    alu_bound_gbs = pipes[mix_name]  # windows/s = bytes/s
    e2e_bound = min(h2d * GB, duplex_in * GB, alu_bound_gbs, d2h * GB * total_bytes / out_bytes) / GB

    out = {
        "metric": METRIC, "value": round(value, 3),
        "value_basis": "hashed GB/s with the inputs resident in HBM (the kernel chain through the C ABI); the "
                       "host-to-digests figure of the metric is e2e.value",
        "device_resident_gbs": round(value, 3), "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dev_ms / args.steps, 4),
        "step_ms_stats": _mean_ci(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": f"sliding-window {args.hash.upper()}, {U} units x {N // 1024} KiB, w=20, "
                               "mask=target=0x1FFF, chunk direct hash S=4 KiB",
                   "units_per_gpu": U, "unit_bytes": N, "window": 20, "mask": 0x1FFF, "target": 0x1FFF,
                   "chunk_segment_bytes": 4096, "content": "50% repeated 8 KiB blocks from a pool of 64",
                   "l2": (f"inputs ({U * N / 2**20:.0f} MiB per step) larger than L2 (126 MB); no flush"
                          if U * N > 126e6 else f"inputs ({U * N / 2**20:.0f} MiB per step) fit in L2 (126 MB); "
                                                  "no flush: a small case, not a bench line"),
                   "parallelism": f"replicas x{ws}", "streams": args.streams, "batch_jobs": args.batch_jobs,
                   "e2e_job_sets": args.e2e_sets,
                   "graphs": bool(args.graphs)},
        "roofline": {"bound": "alu", "kernel": "k_sliding_windows", "achieved": round(achieved, 3),
                     "peak": round(peak, 3), "unit": "Tops/s (int32)", "frac": round(achieved / peak, 4),
                     "peak_basis": "measured: LOP3 and IMAD chains alternating (integer ALU and FMA pipes "
                                   "dual-issuing), crystal_alu_probe, CUDA events, at the sampled clock",
                     "traffic": traffic, "traffic_unit": "bytes per launch (ncu dram read+write)",
                     "ops_per_window": ops_per_window, "windows_per_launch": windows,
                     "avg_launch_ms": round(win_avg_s * 1e3, 4),
                     "window_hash_ceiling": round(mix_ceiling, 3),
                     "frac_of_window_hash_ceiling": round(achieved / mix_ceiling, 4),
                     "window_hash_ceiling_basis": f"measured: the {args.hash.upper()} 20-byte window hash on "
                                                  "register data (crystal_alu_probe), windows/s x ops_per_window",
                     "nominal_issue_peak": round(nominal, 3),
                     "frac_of_nominal_issue_peak": round(achieved / nominal, 4),
                     "nominal_basis": f"{SM_COUNT_B300} SMs x {INT_LANES_PER_SM} int32 lanes/clk x {sm_max:.0f} MHz",
                     "pipes_measured_Tops": {k: round(v / 1e12, 3) for k, v in pipes.items()
                                             if not k.endswith("windows")},
                     "windows_per_s_measured_G": {k: round(v / 1e9, 2) for k, v in pipes.items()
                                                  if k.endswith("windows")}},
        "e2e": None if e2e_value is None else {
            "value": round(e2e_value, 3), "unit": "GB/s", "h2d_bytes_per_step": total_bytes * ws,
            "d2h_bytes_per_step": U * out_size * ws, "ms_per_step": round(e2e_wall * 1e3 / args.steps, 3),
            "step_spacing_ms_stats": _mean_ci(e2e_step_ms) if len(e2e_step_ms) > 1 else None,
            "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3),
                           "p99": round(float(np.percentile(lat, 99)), 3)},
            "roofline_gbs": round(e2e_bound, 2), "frac": round(e2e_value / ws / e2e_bound, 4),
            "roofline_basis": "min(best measured H2D, measured H2D+D2H duplex rate scaled to the input share, "
                              "best measured D2H scaled to the output bytes, measured window-hash ceiling)",
            "copy_only_gbs": round(copy_only, 3),
            "copy_only_note": "the same jobs with the dummy kernel: copy-in and copy-out only"},
        "host_link": link,
        "clocks": clock_info,
        "gpu_launches": int(launches),
        "gpu_launches_split": {"value_region": int(launches_value), "e2e_region": int(launches - launches_value)},
        "wall_s": round(wall, 3),
    }
    out["_gpu_results"] = gpu_results
    if ctx is not None:
        ctx.shutdown()
    if dist is not None:
        dist.destroy_process_group()
    return out


def run_direct_value(args, ws, rank, local):
    """Direct hashing, inputs resident in HBM: segment MD5s + digest of digests
    over ``units`` units of ``unit_bytes`` uniform random bytes (4 KiB
    segments).  Prints its own line; not the headline workload."""
    import torch

    from paper_1005_1695_b300 import crystal as C
    from paper_1005_1695_b300 import inputs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    C.load()
    U, N = args.units, args.unit_bytes
    d_in = torch.empty(U * N, dtype=torch.uint8, device=dev)
    for u in range(U):
        d_in[u * N:(u + 1) * N].copy_(torch.from_numpy(inputs.uniform_unit(args.seed, u, N)))
    p = C.params(segment_bytes=args.segment_bytes)
    batch = C.DeviceBatch(d_in, [u * N for u in range(U)], [N] * U, [C.CRYSTAL_KIND_MD5_DIRECT] * U, p)
    desc_host = torch.from_numpy(batch.host_desc).pin_memory()
    torch.cuda.synchronize()
    stream = torch.cuda.Stream(device=dev)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]

    def step(i=None):
        with torch.cuda.stream(stream):
            batch.d_desc.copy_(desc_host, non_blocking=True)
            if i is not None:
                ev[i][0].record(stream)
            batch.launch_direct_segments(stream)
            if i is not None:
                ev[i][1].record(stream)
            batch.launch_direct_outer(stream)
            if i is not None:
                ev[i][2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for i in range(args.steps):
        step(i)
    torch.cuda.synchronize()
    seg_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
    tot_ms = float(np.mean([e[0].elapsed_time(e[2]) for e in ev]))
    blocks = U * sum(((min(args.segment_bytes, N - o) + 8) // 64 + 1) for o in range(0, N, args.segment_bytes))
    peaks = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6354.7))
    line = {"metric": "direct hashed GB/s, inputs resident in HBM", "value": round(U * N / tot_ms / 1e6, 2),
            "unit": "GB/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(tot_ms, 4), "dtype": "u8", "data": "synthetic", "impl": "ours",
            "config": {"workload": f"direct MD5, {U} units x {N >> 20} MiB, S={args.segment_bytes}"},
            "segments_kernel": {"avg_launch_ms": round(seg_ms, 4), "GB_per_s": round(U * N / seg_ms / 1e6, 1),
                                "hbm_frac": round(U * N / seg_ms / 1e6 / hbm, 4),
                                "compressions_per_s_G": round(blocks / seg_ms / 1e6, 2)},
            "outer_kernel_ms": round(tot_ms - seg_ms, 4)}
    print(json.dumps(line))


# ---- the other configurations, as compact records of the default line -------------

class Checks:
    """Outputs the GPU produced for a seeded sample of a configuration's units
    (at least 1%, always including its largest direct and sliding units),
    with what the oracle needs to recompute them.  The CPU-baseline leg runs
    the oracle on exactly these units: its rate is that record's
    ``cpu_baseline`` and the comparison its ``verified`` record."""

    def __init__(self):
        self.items = []  # (kind, host bytes, out_size, oracle params, GPU used bytes)

    def add(self, kind, data, out_size, got, params=None):
        self.items.append((int(kind), data, int(out_size), params or {}, bytes(got)))

    def run_oracle(self, cores: int):
        import oracle
        from concurrent.futures import ThreadPoolExecutor

        oracle.build()
        order = sorted(range(len(self.items)), key=lambda i: -len(self.items[i][1]))

        def one(i):
            kind, data, osz, prm, got = self.items[i]
            st, want = oracle.task(kind, data, osz, **prm)
            return st in (0, 1) and want[:len(got)] == got and len(got) > 0

        t0 = time.perf_counter()
        with ThreadPoolExecutor(max_workers=cores) as ex:
            ok = list(ex.map(one, order))
        dt = time.perf_counter() - t0
        nbytes = sum(len(x[1]) for x in self.items)
        cpu = {"value": round(nbytes / dt / GB, 4), "unit": "GB/s", "cores": cores, "kind": "oracle",
               "sample": f"the {len(self.items)} checked units ({nbytes / 1e6:.1f} MB), {cores} threads, {dt:.1f} s"}
        ver = {"units_checked": len(ok), "bit_exact": int(sum(ok)), "against": "the oracle, every output byte",
               "largest_checked_bytes": max((len(x[1]) for x in self.items), default=0)}
        return cpu, ver


def _sample(sizes, kinds, every: int):
    """Indices every ``every``-th plus the largest direct and largest sliding unit."""
    from paper_1005_1695_b300 import crystal as C

    idx = set(range(0, len(sizes), every))
    for group in (C.DIRECT_KINDS, C.SLIDING_KINDS):
        cand = [i for i in range(len(sizes)) if int(kinds[i]) in group]
        if cand:
            idx.add(max(cand, key=lambda i: int(sizes[i])))
    return sorted(idx)


def record_config1(args, local, link):
    """64 x 64 KiB, direct hashing, 4 KiB segments: the plain form (per-job
    allocation, one stream, one job at a time) against the pooled,
    overlapped, batched form; every unit checked."""
    from paper_1005_1695_b300 import crystal as C
    from paper_1005_1695_b300 import inputs
    from paper_1005_1695_b300 import streams as S

    U, N = 64, 65536
    p = C.params(segment_bytes=4096)
    units = [inputs.uniform_unit(args.seed, i, N) for i in range(U)]
    rec, checks = {"workload": f"plain direct hashing, {U} units x 64 KiB, S=4 KiB"}, Checks()
    for mode in ("plain", "pooled"):
        runs = [S.run_stream(mode, lambda i: units[i], U, N, C.CRYSTAL_KIND_MD5_DIRECT, p, 16, streams=8,
                             batch_jobs=8, device=local, keep=range(U)) for _ in range(3)]
        r = sorted(runs, key=lambda x: x.seconds)[1]
        assert all(st == 0 for st in r.statuses)
        rec[mode] = {"GB_per_s": round(r.gbs, 3), "latency_ms": {"p50": round(r.latency(50), 3),
                                                                  "p99": round(r.latency(99), 3)}}
        if mode == "pooled":
            for i in range(U):
                checks.add(C.CRYSTAL_KIND_MD5_DIRECT, units[i], 16, r.outputs[i], {"seg_bytes": 4096})
    rec["speedup_pooled_vs_plain"] = round(rec["pooled"]["GB_per_s"] / rec["plain"]["GB_per_s"], 2)
    return rec, checks


def record_config3(args, local, link):
    """Pipelined direct hashing of 4 MiB units (4 KiB segments) over 8 streams:
    pooled jobs resident in pinned memory, the staging ring fed from pageable
    memory by C++ copy threads, one job at a time (no overlap), and per-job
    allocation."""
    import torch

    from paper_1005_1695_b300 import crystal as C
    from paper_1005_1695_b300 import streams as S

    U, N = args.c3_units, 4 << 20
    US = max(U, args.c3_staged_units)
    # units are 4 MiB windows at seeded offsets of a 2 GiB pageable arena
    arena_bytes = 2 << 30
    arena = _arena_pageable(args.seed + 3, arena_bytes)
    offs = (np.arange(US, dtype=np.int64) * 7919 * 4096 + 13 * np.arange(US)) % (arena_bytes - N)
    unit = lambda i: arena[int(offs[i]):int(offs[i]) + N]
    p = C.params(segment_bytes=4096)
    h2d = max(link["h2d_single_gbs"], link["h2d_multi_gbs"])
    memcpy1 = host_memcpy_rate(torch, arena)
    rec = {"workload": f"pipelined direct hashing of 4 MiB units, S=4 KiB, 8 streams x 8 jobs per batch: the "
                       f"staging ring over the configuration's {US} units, the other forms over {U}",
           "host_link_h2d_gbs": h2d}
    checks = Checks()
    # the staging ring needs no memory per unit, so it runs the whole stream;
    # the resident forms hold every unit in pinned memory at once
    modes = [("pooled", U), ("pooled_staged", US), ("no_overlap", U), ("per_job_malloc", min(U, args.malloc_units))]
    for mode, n in modes:
        sample = sorted(set(range(0, n, max(1, n // 8))) | {n - 1})
        r = S.run_stream(mode, unit, n, N, C.CRYSTAL_KIND_MD5_DIRECT, p, 16, streams=8, batch_jobs=8,
                         depth=args.ring_jobs if mode == "pooled_staged" else args.depth,
                         copy_threads=args.stage_threads, device=local, keep=sample)
        assert all(st == 0 for st in r.statuses), (mode, set(r.statuses))
        rec[mode] = {"units": n, "GB_per_s": round(r.gbs, 3), "frac_of_link": round(r.gbs / h2d, 4)}
        if mode in ("pooled", "pooled_staged"):
            for i in sample:
                checks.add(C.CRYSTAL_KIND_MD5_DIRECT, unit(i), 16, r.outputs[i], {"seg_bytes": 4096})
    bound = min(memcpy1 * args.stage_threads, h2d)
    rec["pooled_staged"].update({"copy_threads": args.stage_threads, "ring_jobs": args.ring_jobs,
                                 "memcpy_1thread_gbs": round(memcpy1, 2), "roofline_gbs": round(bound, 2),
                                 "frac_of_roofline": round(rec["pooled_staged"]["GB_per_s"] / bound, 4),
                                 "roofline_basis": "min(one-thread pageable->pinned memcpy x copy threads, H2D)"})
    rec["speedup_pooled_vs_per_job_malloc"] = round(rec["pooled"]["GB_per_s"] / rec["per_job_malloc"]["GB_per_s"], 2)
    rec["speedup_pooled_vs_no_overlap"] = round(rec["pooled"]["GB_per_s"] / rec["no_overlap"]["GB_per_s"], 2)
    return rec, checks


def host_memcpy_rate(torch, src: np.ndarray, piece: int = 256 << 20, rounds: int = 3) -> float:
    """Pageable -> pinned host memcpy GB/s on one thread, best of ``rounds``
    (the pinned buffer is written by one thread first)."""
    pin = torch.empty(piece, dtype=torch.uint8, pin_memory=True).numpy()
    pin[:] = 0
    best = 0.0
    for _ in range(rounds):
        t0 = time.perf_counter()
        np.copyto(pin, src[:piece])
        best = max(best, piece / (time.perf_counter() - t0) / GB)
    del pin
    return best


def _arena_pageable(seed: int, nbytes: int) -> np.ndarray:
    from paper_1005_1695_b300 import inputs

    return inputs.arena(seed, nbytes)


def record_config4(args, local, link):
    """Uneven units (log-uniform 4 KiB - 16 MiB, 80/20 direct/sliding) read in
    place from a page-locked arena, autotuned, replayed as CUDA graphs;
    against the plain single-stream form on a sample."""
    from paper_1005_1695_b300 import autotune as A
    from paper_1005_1695_b300 import crystal as C
    from paper_1005_1695_b300 import inputs
    from paper_1005_1695_b300 import streams as S

    U = args.c4_units
    arena_bytes = 2 << 30
    src = inputs.arena(args.seed + 4, arena_bytes, out=C.page_aligned(arena_bytes))
    req, _ = S.make_batch(args.seed + 4, U, src.nbytes)
    sample = _sample(req["size"], req["kind"], 100)
    req["capture_offset"] = C.NO_CAPTURE
    cap = 0
    for i in sample:
        req["capture_offset"][i] = cap
        cap += int(req["out_size"][i] + 15) // 16 * 16
    capture = np.zeros(cap, dtype=np.uint8)
    pool = 4 << 30
    h2d = max(link["h2d_single_gbs"], link["h2d_multi_gbs"])
    C.host_register(src)
    try:
        tune_req = req[:min(U, 1000)].copy()
        tune_req["capture_offset"] = C.NO_CAPTURE
        shape, table = A.tune(tune_req, src, device_pool_bytes=pool, device=local, streams=(8, 16),
                              batch_jobs=(8, 32), batch_bytes=(64 << 20,), ring_max=(0, 256 << 10, 1 << 20),
                              repeats=1)
        best, gtable = A.tune_geometry(tune_req, src, shape, device_pool_bytes=pool, device=local, repeats=2)
        # the whole workload with the default geometry, then with the tuned one
        st, res, wall_default = A.run_batch(req, src, shape, device_pool_bytes=pool, device=local, capture=capture)
        C.check(st, "crystal_serve")
        st, res, wall = A.run_batch(req, src, best, device_pool_bytes=pool, device=local, capture=capture)
        C.check(st, "crystal_serve")
        plain_n = min(U, args.c4_plain_units)
        plain_req = req[:plain_n].copy()
        plain_req["capture_offset"] = C.NO_CAPTURE
        stp, resp, wallp = A.run_batch(plain_req, src, A.Setting(1, 1, 64 << 20), device_pool_bytes=pool,
                                       device=local, submit_threads=1,
                                       flags=C.CRYSTAL_FLAG_NO_OVERLAP | C.CRYSTAL_FLAG_NO_BATCH)
        C.check(stp, "crystal_serve")
    finally:
        C.host_unregister(src)
    total = float(req["size"].sum())
    gbs = total / (wall / 1e9) / GB
    plain = float(plain_req["size"].sum()) / (wallp / 1e9) / GB
    checks = Checks()
    for i in sample:
        o, n, off = int(req["src_offset"][i]), int(req["size"][i]), int(req["capture_offset"][i])
        checks.add(int(req["kind"][i]), src[o:o + n], int(req["out_size"][i]),
                   capture[off:off + int(res["used_bytes"][i])])
    rec = {"workload": f"{U} units, log-uniform 4 KiB-16 MiB, 80/20 direct/sliding (w=20), inputs read in place "
                       f"from a 2 GiB page-locked arena (or, for small units when the autotuner picks it, copied "
                       f"into an input ring), CUDA graphs, autotuned",
           "GB": round(total / GB, 2), "GB_per_s": round(gbs, 3), "frac_of_link": round(gbs / h2d, 4),
           "chosen": best.as_dict(), "tuning_table": table, "geometry_table": gtable,
           "tuning_sample_units": len(tune_req),
           "default_geometry_GB_per_s": round(total / (wall_default / 1e9) / GB, 3),
           "plain_single_stream": {"units": plain_n, "GB_per_s": round(plain, 3)},
           "speedup_vs_plain": round(gbs / plain, 2)}
    return rec, checks


def record_config5(args, local, link):
    """Open-loop Poisson request streams through crystal_serve: lognormal sizes
    (median 256 KiB, sigma 1.5, cap 64 MiB), 70/30 direct/sliding, inputs read
    in place from a page-locked arena, 8 GiB device pool."""
    from paper_1005_1695_b300 import crystal as C
    from paper_1005_1695_b300 import inputs
    from paper_1005_1695_b300 import streams as S

    arena_bytes = 1 << 30
    src = inputs.arena(args.seed + 5, arena_bytes, out=C.page_aligned(arena_bytes))
    pool = args.pool_bytes
    h2d = max(link["h2d_single_gbs"], link["h2d_multi_gbs"])
    # the host pool holds outputs and the input ring (inputs are read in place
    # from the arena), and the staged inputs of the pageable-source runs
    ctx = C.Context(max_in_bytes=64 << 20, max_out_bytes=C.sliding_out_bytes(64 << 20, 4 * 8192 + 64),
                    device_pool_bytes=pool, host_pool_bytes=4 << 30, n_streams=args.streams, device=local,
                    max_batch_jobs=args.serve_batch_jobs, max_batch_bytes=32 << 20, flags=C.CRYSTAL_FLAG_GRAPHS)
    ring = dict(ring_bytes=args.input_ring, ring_max_request=args.ring_max)
    rec = {"workload": "open-loop Poisson requests, lognormal sizes (median 256 KiB, sigma 1.5, cap 64 MiB), "
                       f"70/30 direct/sliding, {pool >> 30} GiB device pool, {args.streams} streams, "
                       f"{args.serve_batch_jobs} jobs per batch, inputs read in place from a page-locked arena, "
                       + (f"requests up to {args.ring_max >> 10} KiB copied into a {args.input_ring >> 20} MiB "
                          "input ring (merged transfers)" if args.input_ring else "no input ring"),
           "rates_per_s": {}}
    checks = Checks()
    ctx.prepare_graphs()
    C.host_register(src)
    registered = True

    def median_run(req, capture_bytes, pinned=True, threads=args.copy_threads, **kw):
        # near saturation a run either keeps up with the arrivals or drains a
        # backlog after the last one: each rate runs several times and the
        # run with the median throughput is reported, all of them listed
        runs = []
        for _ in range(args.c5_repeats):
            capture = np.zeros(capture_bytes, dtype=np.uint8)
            s0 = ctx.stats()
            st, res, wall = ctx.serve(src, req, capture=capture, copy_threads=threads,
                                      source_pinned=pinned, **kw)
            C.check(st, "crystal_serve")
            runs.append((wall, res, capture, int(ctx.stats().copies_dma - s0.copies_dma)))
        order = sorted(runs, key=lambda r: r[0])
        return order[len(order) // 2], [r[0] for r in runs]

    try:
        warm, _ = S.make_trace(args.seed + 1, 2000, 10000.0, src.nbytes)
        C.check(ctx.serve(src, warm, copy_threads=args.copy_threads, source_pinned=True, **ring)[0],
                "crystal_serve")
        for rate in args.c5_rates:
            n = int(min(args.max_requests, max(args.min_requests, rate * args.seconds)))
            req, _ = S.make_trace(args.seed, n, rate, src.nbytes)
            sample = _sample(req["size"], req["kind"], 100)
            req["capture_offset"] = C.NO_CAPTURE
            cap = 0
            for i in sample:
                req["capture_offset"][i] = cap
                cap += int(req["out_size"][i] + 15) // 16 * 16
            (wall, res, capture, copies), walls = median_run(req, cap, **ring)
            lat = S.latency_ms(req, res)
            total = int(req["size"].sum())
            span = float(req["arrival_ns"][-1]) / 1e9
            gbs = total / (wall / 1e9) / GB
            entry = {
                "requests": n, "offered_GB_per_s": round(total / max(span, 1e-9) / GB, 3),
                "GB_per_s": round(gbs, 3), "frac_of_link": round(gbs / h2d, 4),
                "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3),
                               "p99": round(float(np.percentile(lat, 99)), 3)},
                "runs_GB_per_s": [round(total / (w / 1e9) / GB, 3) for w in walls], "dma_copies": copies}
            if args.input_ring and rate == max(args.c5_rates):
                # the same requests with every input read in place (one transfer each)
                (w0, res0, _, copies0), walls0 = median_run(req, cap)
                lat0 = S.latency_ms(req, res0)
                entry["without_input_ring"] = {
                    "GB_per_s": round(total / (w0 / 1e9) / GB, 3),
                    "latency_ms": {"p50": round(float(np.percentile(lat0, 50)), 3),
                                   "p99": round(float(np.percentile(lat0, 99)), 3)},
                    "runs_GB_per_s": [round(total / (w / 1e9) / GB, 3) for w in walls0], "dma_copies": copies0}
            rec["rates_per_s"][str(int(rate))] = entry
            for i in sample:
                o, nb, off = int(req["src_offset"][i]), int(req["size"][i]), int(req["capture_offset"][i])
                checks.add(int(req["kind"][i]), src[o:o + nb], int(req["out_size"][i]),
                           capture[off:off + int(res["used_bytes"][i])])
            if rate == max(args.c5_rates):
                last = (rate, n, req, cap, total, span, res, capture, sample)
        # the other source mode: the same highest-rate requests from pageable
        # memory, every request's bytes copied by the staging threads (8)
        rate, n, req, cap, total, span, res, capture, sample = last
        C.host_unregister(src)
        registered = False
        (wp, resp, capp, copiesp), wallsp = median_run(req, cap, pinned=False, threads=8, **ring)
        latp = S.latency_ms(req, resp)
        same = all(capp[int(req["capture_offset"][i]):int(req["capture_offset"][i]) + int(resp["used_bytes"][i])]
                   .tobytes() == capture[int(req["capture_offset"][i]):int(req["capture_offset"][i])
                                         + int(res["used_bytes"][i])].tobytes() for i in sample)
        gbs = total / (wp / 1e9) / GB
        rec["pageable_source"] = {
            "rate_per_s": int(rate), "requests": n, "copy_threads": 8, "GB_per_s": round(gbs, 3),
            "frac_of_link": round(gbs / h2d, 4),
            "latency_ms": {"p50": round(float(np.percentile(latp, 50)), 3),
                           "p99": round(float(np.percentile(latp, 99)), 3)},
            "runs_GB_per_s": [round(total / (w / 1e9) / GB, 3) for w in wallsp], "dma_copies": copiesp,
            "sample_outputs_equal_page_locked_run": bool(same)}
    finally:
        ctx.shutdown()
        if registered:
            C.host_unregister(src)
    return rec, checks


def record_overhead(args, local, link):
    sizes = [4096, 65536, 1 << 20, 16 << 20]
    return {"metric": "framework overhead per job (dummy kernel, equal bytes in and out), microseconds",
            "sizes": measure_overhead(local, sizes, 30),
            "paper_context": "slightly under 70 us per job on a 9800 GX2 host (Section 5.1)"}, Checks()


def record_streamlen(args, local, link):
    return {"metric": "GB/s per stream length, 1 MiB direct-hash jobs (Figure 8's shape)",
            "stream_lengths": measure_streamlen(local, args.seed, (1, 2, 4, 10), 3),
            "stream_lengths_sha1": measure_streamlen(local, args.seed, (1, 2, 4, 10), 3,
                                                     kind=3)}, Checks()


def run_config_records(args, local, link):
    """Records of configurations 1, 3, 4 and 5 (GPU part); returns
    {name: (record, checks)}."""
    out = {}
    for name, fn in (("config1_plain", record_config1), ("config3_pipelined", record_config3),
                     ("config4_batched", record_config4), ("config5_served", record_config5),
                     ("sha1_sliding", record_sha1), ("overhead_per_job", record_overhead),
                     ("stream_length", record_streamlen), ("stream_of_10_by_size", record_sizes)):
        t0 = time.perf_counter()
        rec, checks = fn(args, local, link)
        rec["wall_s"] = round(time.perf_counter() - t0, 1)
        out[name] = (rec, checks)
    return out


def _capture_sample(C, req, every: int = 100):
    """Capture slots for a seeded sample of ``req`` (``_sample``); other
    requests are not captured.  Returns the capture buffer."""
    sample = _sample(req["size"], req["kind"], every)
    req["capture_offset"] = C.NO_CAPTURE
    cap = 0
    for i in sample:
        req["capture_offset"][i] = cap
        cap += int(req["out_size"][i] + 15) // 16 * 16
    return np.zeros(max(cap, 16), dtype=np.uint8)


def _add_checks(checks, req, res, src, capture):
    for i in np.nonzero(req["capture_offset"] != np.uint64((1 << 64) - 1))[0]:
        o, n, off = int(req["src_offset"][i]), int(req["size"][i]), int(req["capture_offset"][i])
        checks.add(int(req["kind"][i]), src[o:o + n], int(req["out_size"][i]),
                   capture[off:off + int(res["used_bytes"][i])])


def _verified(args, checks):
    """--verify: the CPU-baseline leg of a single-workload run -- the oracle
    timed on the sampled units and compared with the GPU's outputs."""
    if not args.verify or not checks.items:
        return {}
    cpu, ver = checks.run_oracle(len(os.sched_getaffinity(0)))
    return {"cpu_baseline": cpu, "verified": ver}


def run_stream_modes(args, local, kind, unit_bytes, n_units, modes, subset=None, unit=None):
    """One stream of jobs per mode through the job API; digests of every mode
    must agree.  ``unit(i)`` gives unit i's bytes (default: seeded uniform
    random bytes).  Returns one record per mode (these workloads are not the
    headline)."""
    import torch

    from paper_1005_1695_b300 import crystal as C
    from paper_1005_1695_b300 import inputs
    from paper_1005_1695_b300 import streams as S

    torch.cuda.set_device(local)
    C.load()
    p = C.params(segment_bytes=4096)
    out_size = 16 if kind == C.CRYSTAL_KIND_MD5_DIRECT else C.sliding_out_bytes(unit_bytes, args.max_chunks)

    if unit is None:
        def unit(i):
            return inputs.uniform_unit(args.seed, i, unit_bytes)

    results, outs = {}, {}
    for mode in modes:
        n = n_units if not subset or mode not in subset else min(n_units, subset[mode])
        runs = []
        for _ in range(max(1, args.steps)):
            staged = mode == "pooled_staged"
            r = S.run_stream(mode, unit, n, unit_bytes, kind, p, out_size, streams=args.streams,
                             batch_jobs=args.batch_jobs, depth=args.ring_jobs if staged else args.depth,
                             copy_threads=args.stage_threads, device=local, keep=range(0, n, max(1, n // 32)))
            assert all(st == C.CRYSTAL_OK for st in r.statuses), (mode, set(r.statuses))
            runs.append(r)
        best = sorted(runs, key=lambda r: r.seconds)[len(runs) // 2]  # median run
        results[mode] = {"units": n, "GB_per_s": round(best.gbs, 3), "s": round(best.seconds, 4),
                         "latency_ms": {"p50": round(best.latency(50), 3), "p99": round(best.latency(99), 3)}}
        outs[mode] = best.outputs
    ref = outs[modes[0]]
    for mode in modes[1:]:
        for i, o in outs[mode].items():
            if i in ref:
                assert o == ref[i], f"mode {mode} differs from {modes[0]} on unit {i}"
    if args.verify:  # every mode agrees with the first on these units; the first against the oracle
        checks = Checks()
        for i, o in ref.items():
            checks.add(kind, unit(i), out_size, o, {"seg_bytes": 4096})
        results["_verify"] = _verified(args, checks)
    return results


def run_plain(args, ws, rank, local):
    """64 units of 64 KiB, direct hashing, 4 KiB segments: the plain
    single-stream form against the pooled, overlapped, batched form."""
    from paper_1005_1695_b300 import crystal as C

    U, N = args.units or 64, args.unit_bytes or 65536
    res = run_stream_modes(args, local, C.CRYSTAL_KIND_MD5_DIRECT, N, U, ["plain", "no_overlap", "pooled"])
    print(json.dumps({"metric": "end-to-end hashed GB/s through the job API", "unit": "GB/s",
                      "workload": f"plain direct hashing, {U} units x {N >> 10} KiB, S=4 KiB",
                      "modes": res, "steps": args.steps, "data": "synthetic"}))


def run_pipelined(args, ws, rank, local):
    """Direct hashing of a long stream of 4 MiB units with pooled buffers and
    overlap, against no-overlap and per-job allocation."""
    import torch

    from paper_1005_1695_b300 import crystal as C

    U, N = args.units or 4096, args.unit_bytes or (4 << 20)
    # units are N-byte windows at seeded offsets of a 2 GiB pageable arena
    arena_bytes = 2 << 30
    arena = _arena_pageable(args.seed + 3, arena_bytes)
    offs = (np.arange(U, dtype=np.int64) * 7919 * 4096 + 13 * np.arange(U)) % (arena_bytes - N)
    res = run_stream_modes(args, local, C.CRYSTAL_KIND_MD5_DIRECT, N, U,
                           ["pooled", "no_overlap", "pooled_staged", "per_job_malloc"],
                           subset={"per_job_malloc": args.malloc_units},
                           unit=lambda i: arena[int(offs[i]):int(offs[i]) + N])
    link = measure_link(torch, torch.device("cuda", local), 256 << 20)
    h2d = max(link["h2d_single_gbs"], link["h2d_multi_gbs"])
    ver = res.pop("_verify", {})
    for m in res.values():
        m["frac_of_link"] = round(m["GB_per_s"] / h2d, 4)
    print(json.dumps({"metric": "end-to-end hashed GB/s through the job API", "unit": "GB/s", **ver,
                      "workload": f"pipelined direct hashing, {U} units x {N >> 20} MiB (windows of a 2 GiB "
                                  f"pageable arena), S=4 KiB, {args.streams} streams, {args.batch_jobs} jobs per "
                                  f"batch; staged: {args.stage_threads} copy threads, {args.ring_jobs} ring jobs",
                      "host_link": link, "modes": res, "steps": args.steps,
                      "data": "synthetic"}))


def run_serving(args, ws, rank, local):
    """Open-loop Poisson request streams at several rates through crystal_serve:
    lognormal sizes (median 256 KiB, sigma 1.5, cap 64 MiB), 70/30
    direct/sliding, admission against an 8 GiB device pool."""
    import torch

    from paper_1005_1695_b300 import crystal as C
    from paper_1005_1695_b300 import inputs
    from paper_1005_1695_b300 import streams as S

    torch.cuda.set_device(local)
    C.load()
    src = inputs.arena(args.seed, args.arena_bytes, out=C.page_aligned(args.arena_bytes))
    rates = [float(r) for r in args.rates.split(",")]
    pool = args.pool_bytes
    ctx = C.Context(max_in_bytes=64 << 20, max_out_bytes=C.sliding_out_bytes(64 << 20, 4 * 8192 + 64),
                    device_pool_bytes=pool, host_pool_bytes=pool, n_streams=args.streams, device=local,
                    max_batch_jobs=args.serve_batch_jobs, max_batch_bytes=32 << 20,
                    flags=C.CRYSTAL_FLAG_GRAPHS)
    out = {}
    checks = Checks()
    ctx.prepare_graphs()
    pinned = args.source == "pinned"
    if pinned:
        C.host_register(src)
    try:
        # untimed warm-up: each stream slot captures its graphs and the pools
        # are touched before the first measured rate
        warm, _ = S.make_trace(args.seed + 1, 2000, rates[0], src.nbytes)
        C.check(ctx.serve(src, warm, copy_threads=args.copy_threads, source_pinned=pinned,
                          ring_bytes=args.input_ring, ring_max_request=args.ring_max)[0], "crystal_serve")
        for rate in rates:
            n = int(min(args.max_requests, max(args.min_requests, rate * args.seconds)))
            req, _ = S.make_trace(args.seed, n, rate, src.nbytes)
            capture = _capture_sample(C, req) if args.verify else None
            s0 = ctx.stats()
            st, res, wall = ctx.serve(src, req, copy_threads=args.copy_threads, source_pinned=pinned,
                                      capture=capture, ring_bytes=args.input_ring, ring_max_request=args.ring_max)
            s1 = ctx.stats()
            if args.verify:
                _add_checks(checks, req, res, src, capture)
            ok = res["status"] == 0
            lat = S.latency_ms(req, res)[ok]
            wait = (res["admit_ns"].astype(np.float64) - req["arrival_ns"].astype(np.float64))[ok] / 1e6
            total = int(req["size"][ok].sum())
            span = float(req["arrival_ns"][-1]) / 1e9
            out[f"{int(rate)}"] = {
                "requests": n, "failed": int((~ok).sum()), "GB": round(total / 1e9, 3),
                "offered_GB_per_s": round(float(req["size"].sum()) / max(span, 1e-9) / 1e9, 3),
                "GB_per_s": round(total / (wall / 1e9) / 1e9, 3),
                "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3),
                               "p99": round(float(np.percentile(lat, 99)), 3)},
                "admission_wait_ms_p99": round(float(np.percentile(wait, 99)), 3),
                "batches": int(s1.batches_launched - s0.batches_launched),
                "dma_copies": int(s1.copies_dma - s0.copies_dma),
                "master_issue_busy_frac": round((s1.master_issue_ns - s0.master_issue_ns) / max(wall, 1), 3),
                "master_complete_busy_frac": round((s1.master_complete_ns - s0.master_complete_ns) / max(wall, 1), 3),
                "create_busy_frac": round((s1.create_ns - s0.create_ns) / max(wall, 1), 3),
                "create_calls": int(s1.create_calls - s0.create_calls),
                "create_eagain": int(s1.create_eagain - s0.create_eagain)}
    finally:
        ctx.shutdown()
        if pinned:
            C.host_unregister(src)
    print(json.dumps({"metric": "served hashed GB/s and p50/p99 request latency", "unit": "GB/s",
                      "source": "page-locked, read in place" if pinned else "pageable, staged by copy threads",
                      "workload": "open-loop Poisson requests, lognormal sizes (median 256 KiB, sigma 1.5, "
                                  f"cap 64 MiB), 70/30 direct/sliding, {pool >> 30} GiB device pool, "
                                  f"{args.streams} streams, {args.serve_batch_jobs} jobs per batch, "
                                  f"{args.copy_threads} staging threads, "
                                  + (f"requests up to {args.ring_max >> 10} KiB through a {args.input_ring >> 20} MiB "
                                     "input ring" if args.input_ring else "no input ring"),
                      "rates_per_s": out, "data": "synthetic", **_verified(args, checks)}))


def run_batched(args, ws, rank, local):
    """Uneven units (log-uniform 4 KiB-16 MiB, 80/20 direct/sliding) read in
    place from a page-locked seeded arena, all available at once, packed into
    batches replayed as CUDA graphs with the autotuned setting; against the
    plain single-stream form on a sample."""
    import torch

    from paper_1005_1695_b300 import autotune as A
    from paper_1005_1695_b300 import crystal as C
    from paper_1005_1695_b300 import inputs
    from paper_1005_1695_b300 import streams as S

    torch.cuda.set_device(local)
    C.load()
    src = inputs.arena(args.seed, args.arena_bytes, out=C.page_aligned(args.arena_bytes))
    U = args.units or 100_000
    req, _ = S.make_batch(args.seed, U, src.nbytes)
    pool = args.pool_bytes
    capture = _capture_sample(C, req) if args.verify else None
    checks = Checks()
    C.host_register(src)
    try:
        sample = req[:min(U, args.tune_units)].copy()
        sample["capture_offset"] = C.NO_CAPTURE
        xf = C.CRYSTAL_FLAG_GRAPHS
        shape, table = A.tune(sample, src, device_pool_bytes=pool, device=local, flags=xf,
                              ring_max=(0, 256 << 10, 1 << 20))
        best, gtable = A.tune_geometry(sample, src, shape, device_pool_bytes=pool, device=local, flags=xf)
        st, res, wall = A.run_batch(req, src, best, device_pool_bytes=pool, device=local, flags=xf, capture=capture)
        C.check(st, "crystal_serve")
        if args.verify:
            _add_checks(checks, req, res, src, capture)
        plain_n = min(U, args.malloc_units)
        plain_req = req[:plain_n].copy()
        plain_req["capture_offset"] = C.NO_CAPTURE
        stp, resp, wallp = A.run_batch(plain_req, src, A.Setting(1, 1, 64 << 20), device_pool_bytes=pool,
                                       device=local, submit_threads=1,
                                       flags=C.CRYSTAL_FLAG_NO_OVERLAP | C.CRYSTAL_FLAG_NO_BATCH)
        C.check(stp, "crystal_serve")
    finally:
        C.host_unregister(src)
    link = measure_link(torch, torch.device("cuda", local), 256 << 20)
    h2d = max(link["h2d_single_gbs"], link["h2d_multi_gbs"])
    total = float(req["size"].sum())
    gbs = total / (wall / 1e9) / GB
    print(json.dumps({"metric": "end-to-end hashed GB/s, batched uneven units", "unit": "GB/s",
                      "workload": f"{U} units, log-uniform 4 KiB-16 MiB, 80/20 direct/sliding (w=20), "
                                  f"inputs read in place from a {args.arena_bytes >> 30} GiB page-locked arena "
                                  "(or, for small units when the autotuner picks it, copied into an input ring), "
                                  "CUDA graphs, autotuned",
                      "GB": round(total / GB, 2), "value": round(gbs, 3), "frac_of_link": round(gbs / h2d, 4),
                      "host_link": link, "chosen": best.as_dict(), "tuning_table": table,
                      "geometry_table": gtable, "tuning_sample_units": len(sample),
                      "plain_single_stream": {"units": plain_n,
                                              "GB_per_s": round(float(req["size"][:plain_n].sum()) / (wallp / 1e9) / GB, 3)},
                      "data": "synthetic", **_verified(args, checks)}))


def measure_overhead(local: int, sizes, reps: int) -> dict:
    """Framework overhead of one job (Section 5.1, Figure 5): copy in n bytes,
    dummy kernel, copy out n bytes, issued directly vs through the job
    runtime; the difference is the framework's own cost (medians)."""
    import torch

    from paper_1005_1695_b300 import crystal as C

    torch.cuda.set_device(local)
    L = C.load()
    stream = torch.cuda.Stream()
    out = {}
    with C.Context(max_in_bytes=max(sizes), max_out_bytes=max(sizes), device_pool_bytes=2 * max(sizes) + (64 << 20),
                   host_pool_bytes=2 * max(sizes) + (16 << 20), n_streams=1, device=local) as ctx:
        for n in sizes:
            t = ctx.task_create(n, n)
            # the direct path moves the very same buffers: the job's pinned and device memory
            h_in, h_out = L.crystal_task_host_in(t.handle), L.crystal_task_host_out(t.handle)
            d_in, d_out = L.crystal_task_device_in(t.handle), L.crystal_task_device_out(t.handle)
            raw = []
            for i in range(reps + 5):
                t0 = time.perf_counter()
                C.check(L.crystal_direct_job(h_in, d_in, n, h_out, d_out, n, stream.cuda_stream),
                        "crystal_direct_job")
                if i >= 5:
                    raw.append(time.perf_counter() - t0)
            fw, disp, run = [], [], []
            for i in range(reps + 5):
                t0 = time.perf_counter()
                C.check(t.submit(C.CRYSTAL_KIND_NOP), "submit")
                assert t.wait(10_000_000_000) == C.CRYSTAL_OK
                t1 = time.perf_counter()
                if i >= 5:
                    fw.append(t1 - t0)
                    s_ns, d_ns, e_ns = t.timing()
                    disp.append((d_ns - s_ns) / 1e3)
                    run.append((e_ns - d_ns) / 1e3)
            t.release()
            r, f = float(np.median(raw)) * 1e6, float(np.median(fw)) * 1e6
            out[str(n)] = {"direct_us": round(r, 1), "framework_us": round(f, 1), "overhead_us": round(f - r, 1),
                           "overhead_pct": round(100 * (f - r) / f, 1),
                           "submit_to_dispatch_us": round(float(np.median(disp)), 1),
                           "dispatch_to_done_us": round(float(np.median(run)), 1)}
    return out


def run_overhead(args, ws, rank, local):
    sizes = [int(x) for x in args.sizes.split(",")]
    reps = max(30, args.steps)
    print(json.dumps({"metric": "framework overhead per job (dummy kernel, equal bytes in and out)",
                      "unit": "us", "sizes": measure_overhead(local, sizes, reps), "reps": reps,
                      "paper_context": "slightly under 70 us per job on a 9800 GX2 host (Section 5.1)"}))


def measure_streamlen(local: int, seed: int, lengths, reps: int, kind: int = 1) -> dict:
    """Streams of 1..10 jobs of 1 MiB (direct hashing, Figure 8's shape; the
    paper's runs hash with SHA-1, kind 3): the plain form against no-overlap
    and pooled + overlap, per stream length (median of ``reps`` streams
    each)."""
    import torch

    from paper_1005_1695_b300 import crystal as C
    from paper_1005_1695_b300 import inputs
    from paper_1005_1695_b300 import streams as S

    torch.cuda.set_device(local)
    C.load()
    N = 1 << 20
    p = C.params()
    data = [inputs.uniform_unit(seed, i, N) for i in range(max(lengths))]
    out = {}
    for L in lengths:
        row = {}
        for mode in ("plain", "no_overlap", "pooled"):
            runs = [S.run_stream(mode, lambda i: data[i], L, N, kind, p, C.digest_size(kind), streams=8,
                                 batch_jobs=8, depth=24, device=local).seconds for _ in range(reps)]
            row[mode] = round(L * N / float(np.median(runs)) / GB, 3)
        row["speedup_pooled_vs_plain"] = round(row["pooled"] / row["plain"], 2)
        out[str(L)] = row
    return out


def measure_sizes(local: int, seed: int, sizes, jobs: int, reps: int, kind: int = 3) -> dict:
    """Streams of ``jobs`` direct-hash jobs per data size (Figure 7's shape:
    the paper's stream of 10 SHA-1 jobs over block sizes): the plain form
    (allocation per job, one job at a time), buffer reuse alone (pooled, no
    overlap) and reuse with overlap (pooled, 8 streams), median of ``reps``."""
    import torch

    from paper_1005_1695_b300 import crystal as C
    from paper_1005_1695_b300 import inputs
    from paper_1005_1695_b300 import streams as S

    torch.cuda.set_device(local)
    C.load()
    p = C.params()
    out = {}
    for N in sizes:
        data = [inputs.uniform_unit(seed, i, N) for i in range(jobs)]
        row = {}
        for mode in ("plain", "no_overlap", "pooled"):
            runs = [S.run_stream(mode, lambda i: data[i], jobs, N, kind, p, C.digest_size(kind), streams=8,
                                 batch_jobs=8, depth=24, device=local).seconds for _ in range(reps)]
            row[mode] = round(jobs * N / float(np.median(runs)) / GB, 3)
        row["speedup_reuse"] = round(row["no_overlap"] / row["plain"], 2)
        row["speedup_reuse_overlap"] = round(row["pooled"] / row["plain"], 2)
        out[str(N)] = row
    return out


def record_sizes(args, local, link):
    return {"metric": "GB/s per data size, streams of 10 SHA-1 direct-hash jobs (Figure 7's shape)",
            "sizes": measure_sizes(local, args.seed, (64 << 10, 256 << 10, 1 << 20, 4 << 20, 16 << 20), 10, 3),
            "paper_context": "reuse alone > 6x (small blocks) and > 1.6x (large); with overlap up to 8x and "
                             ">= 3x, on a 9800 GX2 (Section 5.2)"}, Checks()


def run_sizes(args, ws, rank, local):
    print(json.dumps({"metric": "GB/s per data size, streams of 10 SHA-1 direct-hash jobs", "unit": "GB/s",
                      "sizes": measure_sizes(local, args.seed, (16 << 10, 64 << 10, 256 << 10, 1 << 20, 4 << 20,
                                                                16 << 20, 64 << 20), 10, max(3, args.steps)),
                      "data": "synthetic"}))


def run_streamlen(args, ws, rank, local):
    print(json.dumps({"metric": "GB/s per stream length, 1 MiB direct-hash jobs", "unit": "GB/s",
                      "stream_lengths": measure_streamlen(local, args.seed, range(1, 11), max(3, args.steps)),
                      "stream_lengths_sha1": measure_streamlen(local, args.seed, range(1, 11), max(3, args.steps),
                                                               kind=3),
                      "data": "synthetic"}))


def record_sha1(args, local, link):
    """The headline sliding workload with SHA-1, the hash of the paper's own
    runs (Section 5.2): device-resident kernel chain and the job API, the
    window kernel against its ALU-pipe bound (432 ALU-only operations per
    window at the measured single-pipe rate)."""
    import torch

    from paper_1005_1695_b300 import crystal as C

    dev = torch.device("cuda", local)
    U, N = 256, 1 << 20
    KIND = C.CRYSTAL_KIND_SHA1_SLIDING
    p = C.params(window_bytes=20, mask=0x1FFF, target=0x1FFF, chunk_segment_bytes=4096)
    out_size = C.sliding_out_bytes(N, args.max_chunks, KIND)
    host = sliding_workload(args.seed, U, N)
    d_in = torch.from_numpy(host).to(dev)
    batch = C.DeviceBatch(d_in, [u * N for u in range(U)], [N] * U, [KIND] * U, p, out_sizes=[out_size] * U)
    desc_host = torch.from_numpy(batch.host_desc).pin_memory()
    stream = torch.cuda.Stream(device=dev)
    steps = 5
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps + 2)]
    for i in range(steps + 2):
        with torch.cuda.stream(stream):
            batch.d_desc.copy_(desc_host, non_blocking=True)
            ev[i][0].record(stream)
            batch.launch_sliding_windows(stream)
            ev[i][1].record(stream)
            batch.launch_sliding_chunks(stream)
            batch.launch_sliding_digests(stream)
            ev[i][2].record(stream)
    torch.cuda.synchronize()
    assert batch.device_status() == 0
    win_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in ev[2:]]))
    step_ms = float(np.mean([e[0].elapsed_time(e[2]) for e in ev[2:]]))
    got = batch.outputs()
    # the job API: two job sets in turn, as the headline e2e leg
    ctx = C.Context(max_in_bytes=N, max_out_bytes=out_size, device_pool_bytes=2 * U * (N + 2 * out_size) + (256 << 20),
                    host_pool_bytes=2 * U * (N + out_size + 4096) + (16 << 20), n_streams=args.streams,
                    max_batch_jobs=args.batch_jobs, max_batch_bytes=args.batch_jobs * N, device=local,
                    flags=C.CRYSTAL_FLAG_GRAPHS)
    try:
        sets = []
        for _ in range(2):
            tasks = [ctx.task_create(N, out_size) for _ in range(U)]
            for u, t in enumerate(tasks):
                t.h_in[:] = host[u * N:(u + 1) * N]
            sets.append((tasks, ctx.task_array(tasks)))
        for k in range(2):  # warm-up: graphs captured
            C.check(ctx.submit_many(sets[k][1], KIND, p), "submit_many")
        for k in range(2):
            C.check(ctx.wait_many(sets[k][1], 60_000_000_000), "wait_many")
        t0 = time.perf_counter()
        C.check(ctx.submit_many(sets[0][1], KIND, p), "submit_many")
        for i in range(steps):
            if i + 1 < steps:
                C.check(ctx.submit_many(sets[(i + 1) % 2][1], KIND, p), "submit_many")
            C.check(ctx.wait_many(sets[i % 2][1], 60_000_000_000), "wait_many")
        e2e_s = time.perf_counter() - t0
        job_out = [sets[0][0][u].output() for u in range(U)]
    finally:
        ctx.shutdown()
    checks = Checks()
    prm = dict(window=20, mask=0x1FFF, target=0x1FFF, chunk_seg_bytes=4096)
    for u in range(0, U, 16):
        n_chunks = int.from_bytes(got[u][:4], "little")
        used = 8 + 4 * (N // 32) + 24 * n_chunks
        assert job_out[u][:used] == got[u][:used], "job output differs from the device batch output"
        checks.add(KIND, host[u * N:(u + 1) * N], out_size, got[u][:used], prm)
    windows = U * (N - 19)
    alu_pipe = link.get("_alu_pipe_Tops", 0.0)
    bound_wps = alu_pipe * 1e12 / 432 if alu_pipe else None
    h2d = max(link["h2d_single_gbs"], link["h2d_multi_gbs"])
    rec = {"workload": f"sliding-window SHA-1, {U} units x 1 MiB, w=20, mask=target=0x1FFF, chunk direct hash S=4 KiB",
           "device_resident_GB_per_s": round(U * N / step_ms / 1e6, 3),
           "window_kernel_ms": round(win_ms, 4), "windows_per_s_G": round(windows / win_ms / 1e6, 2),
           "e2e_GB_per_s": round(steps * U * N / e2e_s / GB, 3), "e2e_frac_of_h2d": round(steps * U * N / e2e_s / GB / h2d, 4)}
    if bound_wps:
        rec.update({"alu_pipe_bound_windows_per_s_G": round(bound_wps / 1e9, 2),
                    "frac_of_alu_pipe_bound": round(windows / win_ms * 1e3 / bound_wps, 4),
                    "alu_pipe_bound_basis": "measured single-pipe rate (LOP3 chains) / 432 ALU-only operations per "
                                            "window (per step two rotates and the logic op, per schedule word two "
                                            "XORs and a rotate)"})
    return rec, checks


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--units", type=int, default=256)
    ap.add_argument("--unit-bytes", type=int, default=1 << 20)
    ap.add_argument("--max-chunks", type=int, default=1024)
    ap.add_argument("--streams", type=int, default=8)
    ap.add_argument("--batch-jobs", type=int, default=8)
    ap.add_argument("--serve-batch-jobs", type=int, default=16,
                    help="served requests: jobs per batch (16 measured steadier than 8 or 32 near saturation)")
    ap.add_argument("--e2e-sets", type=int, default=2,
                    help="job sets the e2e leg alternates (1: each step waits before the next is submitted)")
    ap.add_argument("--graphs", type=int, default=1)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--cpu-units", type=int, default=0, help="oracle sample units (0: 4 per core, <= 256)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--legs", default="value,e2e", help="value (device-resident) and/or e2e (job API)")
    ap.add_argument("--hash", default="md5", choices=["md5", "sha1"],
                    help="hash of the sliding workload (the headline is MD5)")
    ap.add_argument("--workload", default="sliding", choices=["sliding", "direct", "plain", "pipelined", "serving", "batched", "overhead",
                             "streamlen", "sizes"])
    ap.add_argument("--sizes", default="4096,65536,1048576,16777216,67108864")
    ap.add_argument("--tune-units", type=int, default=4000)
    ap.add_argument("--rates", default="1000,2000,5000,10000,20000,50000")
    ap.add_argument("--seconds", type=float, default=2.0)
    ap.add_argument("--min-requests", type=int, default=2000)
    ap.add_argument("--max-requests", type=int, default=20000)
    ap.add_argument("--arena-bytes", type=int, default=1 << 30)
    ap.add_argument("--pool-bytes", type=int, default=8 << 30)
    ap.add_argument("--copy-threads", type=int, default=0,
                    help="serving: threads that bind or stage each admitted request and submit it "
                         "(0: 4 for a page-locked source, 8 for a pageable one, whose bytes they copy)")
    ap.add_argument("--c5-repeats", type=int, default=5)
    ap.add_argument("--input-ring", type=int, default=256 << 20,
                    help="served requests: bytes of the input ring for small requests (0: none)")
    ap.add_argument("--ring-max", type=int, default=256 << 10,
                    help="served requests: largest request staged through the input ring")
    ap.add_argument("--verify", action="store_true",
                    help="single-workload runs (pipelined, serving, batched): time the oracle on a seeded sample "
                         "of the units (at least 1%%, always the largest) and compare every output byte")
    ap.add_argument("--source", default="pinned", choices=["pinned", "pageable"])
    ap.add_argument("--depth", type=int, default=24, help="jobs in flight for staged / per-job-allocation modes")
    ap.add_argument("--malloc-units", type=int, default=512, help="units for the per-job-allocation modes")
    ap.add_argument("--segment-bytes", type=int, default=4096)
    ap.add_argument("--configs", type=int, default=1,
                    help="add the records of configurations 1, 3, 4 and 5 to the default line (rank 0)")
    ap.add_argument("--c3-units", type=int, default=512)
    ap.add_argument("--c3-staged-units", type=int, default=4096,
                    help="units of the staging-ring form in the configuration-3 record")
    ap.add_argument("--ring-jobs", type=int, default=48, help="staging ring of the pageable-source form")
    ap.add_argument("--stage-threads", type=int, default=16, help="copy threads of the staging ring")
    ap.add_argument("--c4-units", type=int, default=5000)
    ap.add_argument("--c4-plain-units", type=int, default=300)
    ap.add_argument("--c5-rates", default="10000,50000")
    args = ap.parse_args()
    if not args.copy_threads:
        args.copy_threads = 8 if args.source == "pageable" else 4
    ws, rank, local = _dist()
    cores = len(os.sched_getaffinity(0))
    params = dict(window=20, mask=0x1FFF, target=0x1FFF, chunk_seg_bytes=4096)
    cpu_units = args.cpu_units or min(args.units, max(4, 8 * cores))

    if args.impl == "reference":
        if rank != 0:
            return
        host = sliding_workload(args.seed, cpu_units, args.unit_bytes)
        for _ in range(args.warmup):
            cpu_oracle_rate(host, args.unit_bytes, min(cpu_units, cores), cores, params)
        vals, t0 = [], time.perf_counter()
        for _ in range(args.steps):
            vals.append(cpu_oracle_rate(host, args.unit_bytes, cpu_units, cores, params))
        wall = time.perf_counter() - t0
        v = float(np.median([x["value"] for x in vals]))
        line = {"metric": METRIC, "value": round(v, 4), "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(wall * 1e3 / args.steps, 1),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
                "data": "synthetic", "impl": "reference",
                "config": {"workload": f"sliding-window MD5, {args.units} units x {args.unit_bytes // 1024} KiB, "
                                       "w=20, mask=target=0x1FFF, chunk direct hash S=4 KiB",
                           "sample_units_per_step": cpu_units},
                "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": cores, "kind": "oracle",
                                 "sample": vals[0]["sample"]},
                "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if args.workload == "serving":
        run_serving(args, ws, rank, local)
        return
    if args.workload in ("overhead", "streamlen", "sizes"):
        {"overhead": run_overhead, "streamlen": run_streamlen, "sizes": run_sizes}[args.workload](args, ws, rank, local)
        return
    if args.workload == "batched":
        if args.units == 256:
            args.units = 0
        if args.arena_bytes == 1 << 30:
            args.arena_bytes = 8 << 30
        run_batched(args, ws, rank, local)
        return
    if args.workload in ("direct", "plain", "pipelined"):
        if args.workload in ("plain", "pipelined") and args.units == 256 and args.unit_bytes == 1 << 20:
            args.units, args.unit_bytes = 0, 0  # the workload's own sizes
        {"direct": run_direct_value, "plain": run_plain, "pipelined": run_pipelined}[args.workload](
            args, ws, rank, local)
        return
    args.check_units = cpu_units
    args.c5_rates = [float(r) for r in args.c5_rates.split(",")] if isinstance(args.c5_rates, str) else args.c5_rates
    out = run_ours(args, ws, rank, local)
    gpu_results = out.pop("_gpu_results")
    link = dict(out["host_link"])
    link["_alu_pipe_Tops"] = out["roofline"]["pipes_measured_Tops"]["lop3"]  # for the SHA-1 record's bound
    records = run_config_records(args, local, link) if (args.configs and rank == 0) else {}
    if rank == 0:
        if records:
            out["configs"] = {}
            for name, (rec, checks) in records.items():
                if not args.no_cpu_baseline and checks.items:
                    rec["cpu_baseline"], rec["verified"] = checks.run_oracle(cores)
                out["configs"][name] = rec
        if not args.no_cpu_baseline:
            kind = 4 if args.hash == "sha1" else 2
            host = sliding_workload(args.seed, cpu_units, args.unit_bytes)
            cb = cpu_oracle_rate(host, args.unit_bytes, cpu_units, cores, params, kind=kind,
                                 results=gpu_results)
            out["verified"] = cb.pop("_verified")
            out["cpu_baseline"] = cb
            out["cpu_oracle_detail"] = cpu_oracle_detail(host, args.unit_bytes, cores, params)
        print(json.dumps(out))


if __name__ == "__main__":
    main()
