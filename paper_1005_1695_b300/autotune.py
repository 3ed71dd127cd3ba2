"""Autotuner for batched job streams.

Picks, by measuring the workload itself, two levels of the runtime's
settings:

1. the pipeline shape: the number of streams the master thread interleaves
   batches over (the pipeline depth of Section 4.2 / Figure 4), how many
   outstanding jobs and bytes it packs into one batch (one descriptor upload
   and one persistent-kernel chain or graph replay), and up to which size
   units are copied into an input ring so that neighbours' copies merge into
   one transfer (0: none; every unit read in place);
2. for each batch size class (the mean input size of a batch's jobs: under
   64 KiB, 64 KiB to 1 MiB, 1 MiB and up) the kernels' launch geometry:
   threads per CTA and CTAs per SM of the segment-digest kernel, CTAs per SM
   and register budget of the window kernel, and CTAs per SM of the
   chunk-segment kernel (``crystal_set_geometry``).

The segment size stays fixed: it is part of the digest's definition, so
tuning it would change results.  Geometry never changes a result: every
kernel walks its work in a grid-stride loop.

Each candidate runs a sample of the workload through ``crystal_serve`` with
every request arriving at once (the batch-processing case of Section 2.2);
the fastest wins.  The table of every measurement is returned so a run can
record why a setting was chosen.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import crystal as C

# Candidate values of each geometry knob, tried one knob at a time per size
# class (coordinate descent from the defaults; 0 = as many CTAs as fit).
GEOMETRY_KNOBS = (
    ("seg_threads", (128, 64, 256)),
    ("seg_ctas_per_sm", (0, 1, 2, 4)),
    ("win_ctas_per_sm", (0, 2, 4)),
    ("win_registers", (32, 64)),
    ("digest_ctas_per_sm", (0, 2)),
)


# Bytes of the input ring when a setting uses one.
RING_BYTES = 256 << 20


@dataclass
class Setting:
    streams: int
    batch_jobs: int
    batch_bytes: int
    geometry: Dict[int, Dict[str, int]] = field(default_factory=dict)  # size class -> geometry fields
    ring_max: int = 0  # units up to this size go through the input ring (0: no ring)

    def serve_kw(self) -> Dict[str, int]:
        return {"ring_bytes": RING_BYTES if self.ring_max else 0, "ring_max_request": self.ring_max}

    def as_dict(self) -> Dict:
        d = {"streams": self.streams, "batch_jobs": self.batch_jobs, "batch_bytes": self.batch_bytes,
             "ring_max": self.ring_max}
        if self.geometry:
            d["geometry"] = {C.SIZE_CLASS_NAMES[k]: v for k, v in sorted(self.geometry.items())}
        return d


def size_classes(sizes: np.ndarray) -> np.ndarray:
    """Size class of each unit by its own size (a batch of one class has its
    mean in that class)."""
    s = np.asarray(sizes, dtype=np.int64)
    return np.where(s < (64 << 10), 0, np.where(s < (1 << 20), 1, 2))


def _context(req: np.ndarray, setting: Setting, device_pool_bytes: int, device: int, flags: int) -> C.Context:
    max_in = int(req["size"].max())
    max_out = int(req["out_size"].max())
    host_pool = int(req["out_size"].astype(np.int64).sum()) + len(req) * 768 + (64 << 20)
    host_pool = min(host_pool, 2 << 30) + setting.serve_kw()["ring_bytes"]
    ctx = C.Context(max_in_bytes=max_in, max_out_bytes=max_out, device_pool_bytes=device_pool_bytes,
                    host_pool_bytes=host_pool, n_streams=setting.streams, device=device,
                    max_batch_jobs=setting.batch_jobs, max_batch_bytes=setting.batch_bytes, flags=flags)
    for cls, g in setting.geometry.items():
        ctx.set_geometry(cls, C.geometry(**g))
    # graphs captured before the measured run, not by its first batches (a
    # setting with more streams has more slots to capture)
    ctx.prepare_graphs()
    return ctx


def run_batch(req: np.ndarray, source: np.ndarray, setting: Setting, *, device_pool_bytes: int,
              device: int = 0, submit_threads: int = 2, capture: np.ndarray = None, flags: int = C.CRYSTAL_FLAG_GRAPHS):
    """All of ``req`` through crystal_serve at once with ``setting`` (its
    geometry per size class included); ``source`` must be page-locked (jobs
    read their inputs in place).  Returns (status, results, wall_ns)."""
    ctx = _context(req, setting, device_pool_bytes, device, flags)
    try:
        return ctx.serve(source, req, copy_threads=submit_threads, source_pinned=True, capture=capture,
                         **setting.serve_kw())
    finally:
        ctx.shutdown()


def tune(req_sample: np.ndarray, source: np.ndarray, *, device_pool_bytes: int, device: int = 0,
         streams: Sequence[int] = (4, 8, 16), batch_jobs: Sequence[int] = (8, 32, 128),
         batch_bytes: Sequence[int] = (32 << 20, 128 << 20), ring_max: Sequence[int] = (0,), repeats: int = 2,
         flags: int = C.CRYSTAL_FLAG_GRAPHS):
    """Measure every pipeline shape on ``req_sample``; return (best, table)."""
    total = float(req_sample["size"].sum())
    table: List[Dict] = []
    for s, j, b, r in itertools.product(streams, batch_jobs, batch_bytes, ring_max):
        setting = Setting(s, j, b, ring_max=r)
        walls = []
        for _ in range(repeats):
            st, res, wall = run_batch(req_sample, source, setting, device_pool_bytes=device_pool_bytes,
                                      device=device, flags=flags)
            C.check(st, "crystal_serve")
            walls.append(wall)
        table.append({**setting.as_dict(), "GB_per_s": round(total / (min(walls) / 1e9) / 1e9, 3)})
    best = max(table, key=lambda r: r["GB_per_s"])
    return Setting(best["streams"], best["batch_jobs"], best["batch_bytes"], ring_max=best["ring_max"]), table


def tune_geometry(req_sample: np.ndarray, source: np.ndarray, setting: Setting, *, device_pool_bytes: int,
                  device: int = 0, repeats: int = 2, min_units: int = 8, margin: float = 0.02,
                  knobs=GEOMETRY_KNOBS, flags: int = C.CRYSTAL_FLAG_GRAPHS):
    """Per size class present in ``req_sample`` (at least ``min_units`` units),
    coordinate descent over the geometry knobs on one context with
    ``setting``'s pipeline shape: each knob's values in turn, keeping a change
    only if it is faster by more than ``margin``.  Returns (setting with the
    chosen geometry, table)."""
    classes = size_classes(req_sample["size"])
    ctx = _context(req_sample, Setting(setting.streams, setting.batch_jobs, setting.batch_bytes,
                                       ring_max=setting.ring_max), device_pool_bytes, device, flags)
    kw = setting.serve_kw()
    table: List[Dict] = []
    chosen: Dict[int, Dict[str, int]] = {}
    try:
        for cls in range(C.CRYSTAL_SIZE_CLASSES):
            sub = req_sample[classes == cls]
            if len(sub) < min_units:
                continue
            total = float(sub["size"].sum())

            def measure(g: Dict[str, int]) -> float:
                ctx.set_geometry(cls, C.geometry(**g))
                C.check(ctx.serve(source, sub, copy_threads=2, source_pinned=True, **kw)[0], "crystal_serve")  # capture
                walls = []
                for _ in range(repeats):
                    st, res, wall = ctx.serve(source, sub, copy_threads=2, source_pinned=True, **kw)
                    C.check(st, "crystal_serve")
                    walls.append(wall)
                gbs = total / (min(walls) / 1e9) / 1e9
                table.append({"size_class": C.SIZE_CLASS_NAMES[cls], "units": len(sub), **g,
                              "GB_per_s": round(gbs, 3)})
                return gbs

            current: Dict[str, int] = {}
            best = measure(current)
            for name, values in knobs:
                for v in values:
                    cand = {**current, name: v}
                    if cand.get(name) == current.get(name, values[0]):
                        continue
                    gbs = measure(cand)
                    if gbs > best * (1 + margin):
                        best, current = gbs, cand
            ctx.set_geometry(cls, C.geometry(**current))
            chosen[cls] = ctx.get_geometry(cls).as_dict()
    finally:
        ctx.shutdown()
    return Setting(setting.streams, setting.batch_jobs, setting.batch_bytes, chosen, ring_max=setting.ring_max), table
