"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no hashing arithmetic: it only draws bytes, sizes and
arrival times.  Both the GPU path's tests/benchmarks and the CPU oracle's
checks take their inputs from here, so a unit is reproducible from
``(seed, unit index)`` alone.

Every stream is numpy's Philox-4x64 counter-based generator keyed by
``(seed, tag, index)``; no global random state is touched.

Workload shapes (the paper measures a stream of data blocks hashed by
StoreGPU, Section 5.2; sizes follow the benchmark configurations):

* ``uniform_unit``  -- uniform random bytes.
* ``dedup_unit``    -- 8 KiB slots, each either fresh random bytes or a copy
  of one of 64 seeded pool blocks (Bernoulli 0.5), so half the content
  repeats, as content-addressable storage sees it.
* ``loguniform_sizes`` / ``lognormal_sizes`` / ``poisson_arrivals`` -- size
  and arrival mixes for the batched and served streams.
"""
from __future__ import annotations

from typing import Optional

import numpy as np

TAG_UNIFORM = 1
TAG_DEDUP_CHOICE = 2
TAG_DEDUP_POOL = 3
TAG_DEDUP_FRESH = 4
TAG_SIZES = 5
TAG_ARRIVALS = 6
TAG_KINDS = 7
TAG_ARENA = 8

MASK64 = (1 << 64) - 1


def rng(seed: int, tag: int, index: int = 0) -> np.random.Generator:
    """Philox generator keyed by ``(seed, tag, index)``."""
    key = np.array([((seed & 0xFFFFFFFF) << 32 | (tag & 0xFFFFFFFF)) & MASK64, index & MASK64],
                   dtype=np.uint64)
    return np.random.Generator(np.random.Philox(key=key))


def uniform_unit(seed: int, unit: int, n: int, out: Optional[np.ndarray] = None) -> np.ndarray:
    """``n`` uniform random bytes for unit ``unit``."""
    b = np.frombuffer(rng(seed, TAG_UNIFORM, unit).bytes(n), dtype=np.uint8)
    if out is None:
        return b.copy()
    out[:n] = b
    return out


def dedup_pool(seed: int, blocks: int = 64, block_bytes: int = 8192) -> np.ndarray:
    """The seeded pool of repeated blocks, shape ``(blocks, block_bytes)``."""
    return np.frombuffer(rng(seed, TAG_DEDUP_POOL, 0).bytes(blocks * block_bytes),
                         dtype=np.uint8).reshape(blocks, block_bytes)


def dedup_unit(seed: int, unit: int, n: int, pool: Optional[np.ndarray] = None,
               slot_bytes: int = 8192, p_repeat: float = 0.5,
               out: Optional[np.ndarray] = None) -> np.ndarray:
    """Unit of ``n`` bytes made of ``slot_bytes`` slots; each slot is a copy of
    a uniformly chosen pool block with probability ``p_repeat``, else fresh
    random bytes.  A final partial slot takes the prefix of its block."""
    if pool is None:
        pool = dedup_pool(seed, block_bytes=slot_bytes)
    slots = (n + slot_bytes - 1) // slot_bytes
    g = rng(seed, TAG_DEDUP_CHOICE, unit)
    repeat = g.random(slots) < p_repeat
    which = g.integers(0, pool.shape[0], size=slots)
    fresh = np.frombuffer(rng(seed, TAG_DEDUP_FRESH, unit).bytes(slots * slot_bytes), dtype=np.uint8)
    buf = fresh.reshape(slots, slot_bytes).copy()
    buf[repeat] = pool[which[repeat]]
    flat = buf.reshape(-1)[:n]
    if out is None:
        return flat.copy()
    out[:n] = flat
    return out


def loguniform_sizes(seed: int, count: int, lo: int = 4096, hi: int = 16 << 20) -> np.ndarray:
    """``count`` sizes, log-uniform on ``[lo, hi]`` bytes (int64)."""
    g = rng(seed, TAG_SIZES, 0)
    x = np.exp(g.uniform(np.log(lo), np.log(hi), size=count))
    return np.clip(np.round(x), lo, hi).astype(np.int64)


def lognormal_sizes(seed: int, count: int, median: int = 256 << 10, sigma: float = 1.5,
                    cap: int = 64 << 20, floor: int = 1) -> np.ndarray:
    """``count`` sizes, lognormal with the given median and sigma, capped."""
    g = rng(seed, TAG_SIZES, 1)
    x = np.exp(np.log(median) + sigma * g.standard_normal(count))
    return np.clip(np.round(x), floor, cap).astype(np.int64)


def poisson_arrivals(seed: int, count: int, rate_per_s: float) -> np.ndarray:
    """Arrival times (seconds from 0) of an open-loop Poisson process."""
    g = rng(seed, TAG_ARRIVALS, int(rate_per_s))
    return np.cumsum(g.exponential(1.0 / rate_per_s, size=count))


def kind_mix(seed: int, count: int, p_sliding: float) -> np.ndarray:
    """Boolean array: True where the job is sliding-window, else direct."""
    return rng(seed, TAG_KINDS, 0).random(count) < p_sliding


def arena(seed: int, nbytes: int, out: Optional[np.ndarray] = None, chunk: int = 1 << 26) -> np.ndarray:
    """A large seeded byte arena, generated in 64 MiB pieces keyed by index."""
    if out is None:
        out = np.empty(nbytes, dtype=np.uint8)
    for i, off in enumerate(range(0, nbytes, chunk)):
        m = min(chunk, nbytes - off)
        out[off:off + m] = np.frombuffer(rng(seed, TAG_ARENA, i).bytes(m), dtype=np.uint8)
    return out
