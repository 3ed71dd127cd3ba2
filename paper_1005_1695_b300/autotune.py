"""Autotuner for batched job streams.

Picks the runtime's launch geometry for a workload by measuring it: the
number of streams the master thread interleaves batches over (the pipeline
depth of Section 4.2 / Figure 4), and how many outstanding jobs and bytes it
packs into one batch (one descriptor upload and one persistent-kernel chain
or graph replay).  The segment size stays fixed: it is part of the digest's
definition, so tuning it would change results.

Each candidate runs the same sample of the workload through ``crystal_serve``
with every request arriving at once (the batch-processing case of
Section 2.2); the fastest wins.  The table of every measurement is returned
so a run can record why a setting was chosen.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass
from typing import Dict, List, Sequence

import numpy as np

from . import crystal as C


@dataclass
class Setting:
    streams: int
    batch_jobs: int
    batch_bytes: int

    def as_dict(self) -> Dict[str, int]:
        return {"streams": self.streams, "batch_jobs": self.batch_jobs, "batch_bytes": self.batch_bytes}


def run_batch(req: np.ndarray, source: np.ndarray, setting: Setting, *, device_pool_bytes: int,
              device: int = 0, submit_threads: int = 2, capture: np.ndarray = None, flags: int = C.CRYSTAL_FLAG_GRAPHS):
    """All of ``req`` through crystal_serve at once with ``setting``; ``source``
    must be page-locked (jobs read their inputs in place).  Returns
    (status, results, wall_ns)."""
    max_in = int(req["size"].max())
    max_out = int(req["out_size"].max())
    host_pool = int(req["out_size"].astype(np.int64).sum()) + len(req) * 512 + (64 << 20)
    ctx = C.Context(max_in_bytes=max_in, max_out_bytes=max_out, device_pool_bytes=device_pool_bytes,
                    host_pool_bytes=min(host_pool, 2 << 30), n_streams=setting.streams, device=device,
                    max_batch_jobs=setting.batch_jobs, max_batch_bytes=setting.batch_bytes, flags=flags)
    try:
        return ctx.serve(source, req, copy_threads=submit_threads, source_pinned=True, capture=capture)
    finally:
        ctx.shutdown()


def tune(req_sample: np.ndarray, source: np.ndarray, *, device_pool_bytes: int, device: int = 0,
         streams: Sequence[int] = (4, 8, 16), batch_jobs: Sequence[int] = (8, 32, 128),
         batch_bytes: Sequence[int] = (32 << 20, 128 << 20), repeats: int = 2, flags: int = C.CRYSTAL_FLAG_GRAPHS):
    """Measure every combination on ``req_sample``; return (best, table)."""
    total = float(req_sample["size"].sum())
    table: List[Dict] = []
    for s, j, b in itertools.product(streams, batch_jobs, batch_bytes):
        setting = Setting(s, j, b)
        walls = []
        for _ in range(repeats):
            st, res, wall = run_batch(req_sample, source, setting, device_pool_bytes=device_pool_bytes,
                                      device=device, flags=flags)
            C.check(st, "crystal_serve")
            walls.append(wall)
        table.append({**setting.as_dict(), "GB_per_s": round(total / (min(walls) / 1e9) / 1e9, 3)})
    best = max(table, key=lambda r: r["GB_per_s"])
    return Setting(best["streams"], best["batch_jobs"], best["batch_bytes"]), table
