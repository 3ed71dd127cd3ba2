"""ctypes binding of ``libcrystal.so`` (the C ABI in ``include/crystal.h``).

Argument marshalling only: every step of the hashing path runs in the
library's CUDA kernels and its C++ runtime.  The function names are the C
names.  PyTorch is used for device memory and stream handles only (see
:class:`DeviceBatch`).

Loading fails loudly if the library cannot be found or built; there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build

CRYSTAL_OK = 0
CRYSTAL_PENDING = 1
CRYSTAL_EINVAL = -1
CRYSTAL_EAGAIN = -2
CRYSTAL_ENOMEM = -3
CRYSTAL_ETIMEDOUT = -4
CRYSTAL_EOVERFLOW = -5
CRYSTAL_ESHUTDOWN = -6
CRYSTAL_EDEVICE = -7

CRYSTAL_KIND_NOP = 0
CRYSTAL_KIND_MD5_DIRECT = 1
CRYSTAL_KIND_MD5_SLIDING = 2
CRYSTAL_KIND_SHA1_DIRECT = 3
CRYSTAL_KIND_SHA1_SLIDING = 4
DIRECT_KINDS = (CRYSTAL_KIND_MD5_DIRECT, CRYSTAL_KIND_SHA1_DIRECT)
SLIDING_KINDS = (CRYSTAL_KIND_MD5_SLIDING, CRYSTAL_KIND_SHA1_SLIDING)


def digest_size(kind: int) -> int:
    return 20 if kind in (CRYSTAL_KIND_SHA1_DIRECT, CRYSTAL_KIND_SHA1_SLIDING) else 16

CRYSTAL_FLAG_NO_POOL = 1
CRYSTAL_FLAG_NO_OVERLAP = 2
CRYSTAL_FLAG_NO_BATCH = 4
CRYSTAL_FLAG_GRAPHS = 8

CRYSTAL_PROBE_MD5_WINDOWS = 0
CRYSTAL_PROBE_SHA1_WINDOWS = 1
CRYSTAL_PROBE_LOP3 = 2
CRYSTAL_PROBE_SHF = 3
CRYSTAL_PROBE_IADD3 = 4
CRYSTAL_PROBE_IMAD = 5
CRYSTAL_PROBE_LOP3_IMAD = 6
PROBE_KINDS = {"md5_windows": 0, "sha1_windows": 1, "lop3": 2, "shf": 3, "iadd3": 4, "imad": 5, "lop3_imad": 6}



class crystal_config(ctypes.Structure):
    _fields_ = [
        ("max_in_bytes", ctypes.c_uint64),
        ("max_out_bytes", ctypes.c_uint64),
        ("device_pool_bytes", ctypes.c_uint64),
        ("host_pool_bytes", ctypes.c_uint64),
        ("device_arena", ctypes.c_void_p),
        ("n_streams", ctypes.c_int32),
        ("device", ctypes.c_int32),
        ("flags", ctypes.c_uint32),
        ("max_batch_jobs", ctypes.c_uint32),
        ("max_batch_bytes", ctypes.c_uint64),
    ]


class crystal_hash_params(ctypes.Structure):
    _fields_ = [
        ("segment_bytes", ctypes.c_uint32),
        ("window_bytes", ctypes.c_uint32),
        ("mask", ctypes.c_uint32),
        ("target", ctypes.c_uint32),
        ("chunk_segment_bytes", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
    ]


class crystal_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "jobs_completed", "batches_launched", "device_pool_bytes", "device_pool_used",
        "host_pool_bytes", "host_pool_used", "jobs_outstanding", "jobs_running", "copies_dma",
        "master_issue_ns", "master_complete_ns", "create_ns", "create_calls", "create_eagain", "graph_captures")]


UNIT_DTYPE = np.dtype([
    ("in", "<u8"), ("n", "<u8"), ("out", "<u8"), ("scratch", "<u8"), ("work_begin", "<u8"),
    ("out_cap", "<u4"), ("seg_bytes", "<u4"), ("window", "<u2"), ("kind", "<u2"), ("mask", "<u4"),
    ("target", "<u4"), ("seg_base", "<u4"),
])
assert UNIT_DTYPE.itemsize == 64
BATCH_HEADER_BYTES = 64

crystal_callback = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p)

REQUEST_DTYPE = np.dtype([("arrival_ns", "<u8"), ("src_offset", "<u8"), ("size", "<u8"), ("out_size", "<u8"),
                          ("capture_offset", "<u8"), ("kind", "<i4"), ("reserved", "<u4")])
RESULT_DTYPE = np.dtype([("status", "<i4"), ("reserved", "<u4"), ("admit_ns", "<u8"), ("submit_ns", "<u8"),
                         ("done_ns", "<u8"), ("used_bytes", "<u8")])
assert REQUEST_DTYPE.itemsize == 48 and RESULT_DTYPE.itemsize == 40
NO_CAPTURE = (1 << 64) - 1


CRYSTAL_TASK_EXTERNAL_INPUT = 1
CRYSTAL_SERVE_SOURCE_PINNED = 1
CRYSTAL_SERVE_ARRIVAL_ORDER = 2


class crystal_geometry(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in ("seg_threads", "seg_ctas_per_sm", "win_ctas_per_sm", "win_registers",
                                               "digest_ctas_per_sm", "reserved")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_ if n != "reserved"}


CRYSTAL_SIZE_CLASSES = 3
SIZE_CLASS_NAMES = ("under 64 KiB", "64 KiB to 1 MiB", "1 MiB and up")


def geometry(**kw) -> crystal_geometry:
    g = crystal_geometry()
    for k, v in kw.items():
        setattr(g, k, int(v))
    return g


class crystal_stream_config(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("copy_threads", ctypes.c_uint32), ("ring_jobs", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("out_size", ctypes.c_uint64), ("params", ctypes.c_void_p)]


class crystal_serve_config(ctypes.Structure):
    _fields_ = [("copy_threads", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("direct_params", ctypes.c_void_p), ("sliding_params", ctypes.c_void_p),
                ("capture", ctypes.c_void_p), ("capture_bytes", ctypes.c_uint64), ("bypass_ns", ctypes.c_uint64),
                ("ring_bytes", ctypes.c_uint64), ("ring_max_request", ctypes.c_uint64)]

_lib = None
_u64 = ctypes.c_uint64
_vp = ctypes.c_void_p


def lib_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Load (building first if the sources are newer) ``libcrystal.so``."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError("libcrystal.so is missing and could not be built")
    L = ctypes.CDLL(path)
    sig = {
        "crystal_config_default": (None, [ctypes.POINTER(crystal_config)]),
        "crystal_params_default": (None, [ctypes.POINTER(crystal_hash_params)]),
        "crystal_init": (ctypes.c_int, [ctypes.POINTER(crystal_config), ctypes.POINTER(_vp)]),
        "crystal_shutdown": (ctypes.c_int, [_vp]),
        "crystal_task_create": (ctypes.c_int, [_vp, _u64, _u64, ctypes.POINTER(_vp)]),
        "crystal_task_host_in": (_vp, [_vp]),
        "crystal_task_host_out": (_vp, [_vp]),
        "crystal_task_device_in": (_u64, [_vp]),
        "crystal_task_device_out": (_u64, [_vp]),
        "crystal_task_resize": (ctypes.c_int, [_vp, _u64, _u64]),
        "crystal_task_submit": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(crystal_hash_params),
                                               crystal_callback, _vp]),
        "crystal_task_submit_many": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_uint32, ctypes.c_int,
                                                    ctypes.POINTER(crystal_hash_params), crystal_callback, _vp]),
        "crystal_task_poll": (ctypes.c_int, [_vp]),
        "crystal_task_set_priority": (ctypes.c_int, [_vp, ctypes.c_int]),
        "crystal_task_create_ex": (ctypes.c_int, [_vp, _u64, _u64, _u64, ctypes.c_uint32, ctypes.POINTER(_vp)]),
        "crystal_task_bind_input": (ctypes.c_int, [_vp, _vp, _u64]),
        "crystal_host_register": (ctypes.c_int, [_vp, _u64]),
        "crystal_host_unregister": (ctypes.c_int, [_vp]),
        "crystal_serve": (ctypes.c_int, [_vp, _vp, _u64, _vp, ctypes.c_uint32, ctypes.POINTER(crystal_serve_config),
                                         _vp, ctypes.POINTER(_u64)]),
        "crystal_stream_staged": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_uint32, ctypes.POINTER(crystal_stream_config),
                                                 _vp, _u64, _vp, ctypes.POINTER(_u64)]),
        "crystal_get_config": (ctypes.c_int, [_vp, ctypes.POINTER(crystal_config)]),
        "crystal_set_geometry": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(crystal_geometry)]),
        "crystal_get_geometry": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(crystal_geometry)]),
        "crystal_task_wait": (ctypes.c_int, [_vp, ctypes.c_int64]),
        "crystal_task_release": (ctypes.c_int, [_vp]),
        "crystal_task_timing": (ctypes.c_int, [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64),
                                               ctypes.POINTER(_u64)]),
        "crystal_task_wait_many": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_uint32, ctypes.c_int64]),
        "crystal_task_timing_many": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_uint32, _vp]),
        "crystal_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(crystal_stats)]),
        "crystal_prepare_graphs": (ctypes.c_int, [_vp]),
        "crystal_out_bytes": (_u64, [ctypes.c_int, _u64, ctypes.POINTER(crystal_hash_params)]),
        "crystal_sliding_out_bytes": (_u64, [_u64, _u64]),
        "crystal_out_bytes_for_chunks": (_u64, [ctypes.c_int, _u64, _u64]),
        "crystal_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "crystal_kernel_launches": (_u64, []),
        "crystal_direct_job": (ctypes.c_int, [_vp, _vp, _u64, _vp, _vp, _u64, _vp]),
        "crystal_alu_probe": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _vp,
                                             _vp, ctypes.POINTER(_u64)]),
        "crystal_scratch_bytes": (_u64, [ctypes.c_int, _u64, _u64, ctypes.POINTER(crystal_hash_params)]),
        "crystal_batch_plan": (ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.c_uint32]),
        "crystal_batch_bytes": (_u64, [ctypes.c_uint32]),
        "crystal_arena_create": (ctypes.c_int, [_u64, _u64, ctypes.POINTER(_vp)]),
        "crystal_arena_alloc": (ctypes.c_int, [_vp, _u64, ctypes.POINTER(_u64)]),
        "crystal_arena_alloc_at": (ctypes.c_int, [_vp, _u64, ctypes.c_int, ctypes.POINTER(_u64)]),
        "crystal_arena_alloc_exact": (ctypes.c_int, [_vp, _u64, _u64]),
        "crystal_arena_free": (ctypes.c_int, [_vp, _u64]),
        "crystal_arena_used": (_u64, [_vp]),
        "crystal_arena_largest_free": (_u64, [_vp]),
        "crystal_arena_destroy": (None, [_vp]),
    }
    for name in ("crystal_launch_direct", "crystal_launch_direct_segments", "crystal_launch_direct_outer",
                 "crystal_launch_sliding", "crystal_launch_sliding_windows", "crystal_launch_sliding_chunks",
                 "crystal_launch_sliding_digests", "crystal_launch_batch"):
        sig[name] = (ctypes.c_int, [_vp, _vp])
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(status: int, what: str = "") -> int:
    """``status`` if it is not an error, else raise CrystalError (a
    RuntimeError carrying the status)."""
    if status < 0:
        raise CrystalError(status, what)
    return status


def params(segment_bytes=4096, window_bytes=20, mask=0x1FFF, target=0x1FFF, chunk_segment_bytes=4096):
    return crystal_hash_params(segment_bytes, window_bytes, mask, target, chunk_segment_bytes, 0)


def out_bytes(kind: int, in_size: int, p: Optional[crystal_hash_params] = None) -> int:
    return int(load().crystal_out_bytes(kind, in_size, ctypes.byref(p) if p is not None else None))


def sliding_out_bytes(in_size: int, max_chunks: int, kind: int = CRYSTAL_KIND_MD5_SLIDING) -> int:
    return int(load().crystal_out_bytes_for_chunks(kind, in_size, max_chunks))


def scratch_bytes(kind: int, n: int, out_size: int, p: Optional[crystal_hash_params] = None) -> int:
    return int(load().crystal_scratch_bytes(kind, n, out_size, ctypes.byref(p) if p is not None else None))


def kernel_launches() -> int:
    return int(load().crystal_kernel_launches())


def page_aligned(nbytes: int) -> np.ndarray:
    """A uint8 array whose data starts on a 4 KiB page (for host_register)."""
    raw = np.empty(nbytes + 4096, dtype=np.uint8)
    off = (-raw.ctypes.data) % 4096
    return raw[off:off + nbytes]


def host_register(arr: np.ndarray) -> None:
    """Page-lock ``arr``'s memory (crystal_host_register)."""
    check(load().crystal_host_register(arr.ctypes.data, arr.nbytes), "crystal_host_register")


def host_unregister(arr: np.ndarray) -> None:
    check(load().crystal_host_unregister(arr.ctypes.data), "crystal_host_unregister")


# ---- job runtime ---------------------------------------------------------------

class Task:
    """One job (Figure 2's job_t): numpy views of the pinned host buffers."""

    def __init__(self, ctx: "Context", handle: int, in_size: int, out_size: int):
        self.ctx, self.handle = ctx, handle
        self.in_size, self.out_size = in_size, out_size
        L = load()
        hin, hout = L.crystal_task_host_in(handle), L.crystal_task_host_out(handle)
        self.h_in = np.ctypeslib.as_array((ctypes.c_uint8 * max(in_size, 1)).from_address(hin))[:in_size] \
            if hin else np.zeros(0, np.uint8)
        self.h_out = np.ctypeslib.as_array((ctypes.c_uint8 * max(out_size, 1)).from_address(hout))[:out_size] \
            if hout else np.zeros(0, np.uint8)

    def bind_input(self, arr: Optional[np.ndarray]):
        """crystal_task_bind_input: read the next submit's input from ``arr``
        (keep it alive and unchanged until the job completes)."""
        if arr is None:
            check(load().crystal_task_bind_input(self.handle, None, 0), "crystal_task_bind_input")
            return
        self._bound = arr
        check(load().crystal_task_bind_input(self.handle, arr.ctypes.data, arr.nbytes), "crystal_task_bind_input")
        self.in_size = arr.nbytes

    def resize(self, in_size: int, out_size: int):
        check(load().crystal_task_resize(self.handle, in_size, out_size), "crystal_task_resize")
        self.in_size, self.out_size = in_size, out_size

    def submit(self, kind: int, p: Optional[crystal_hash_params] = None, callback=None, user=None) -> int:
        cb = callback if callback is not None else crystal_callback()
        self._cb_keepalive = cb
        return load().crystal_task_submit(self.handle, kind, ctypes.byref(p) if p is not None else None, cb, user)

    def set_priority(self, priority: int) -> int:
        return load().crystal_task_set_priority(self.handle, priority)

    def poll(self) -> int:
        return load().crystal_task_poll(self.handle)

    def wait(self, timeout_ns: int = -1) -> int:
        return load().crystal_task_wait(self.handle, timeout_ns)

    def release(self) -> int:
        st = load().crystal_task_release(self.handle)
        if st == CRYSTAL_OK:
            self.ctx._tasks.discard(self)
        return st

    def timing(self):
        a, b, c = _u64(), _u64(), _u64()
        check(load().crystal_task_timing(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def output(self, n: Optional[int] = None) -> bytes:
        return self.h_out[: self.out_size if n is None else n].tobytes()


class Context:
    """init(...) / finalize() of Figure 3 as a Python object."""

    def __init__(self, max_in_bytes=64 << 20, max_out_bytes=16 << 20, device_pool_bytes=1 << 30,
                 host_pool_bytes=512 << 20, n_streams=4, device=0, flags=0, max_batch_jobs=64,
                 max_batch_bytes=32 << 20, device_arena=None):
        L = load()
        cfg = crystal_config()
        L.crystal_config_default(ctypes.byref(cfg))
        cfg.max_in_bytes, cfg.max_out_bytes = max_in_bytes, max_out_bytes
        cfg.device_pool_bytes, cfg.host_pool_bytes = device_pool_bytes, host_pool_bytes
        cfg.n_streams, cfg.device, cfg.flags = n_streams, device, flags
        cfg.max_batch_jobs, cfg.max_batch_bytes = max_batch_jobs, max_batch_bytes
        self._arena_ref = device_arena
        if device_arena is not None:
            cfg.device_arena = device_arena.data_ptr()
            cfg.device_pool_bytes = device_arena.numel() * device_arena.element_size()
        h = _vp()
        check(L.crystal_init(ctypes.byref(cfg), ctypes.byref(h)), "crystal_init")
        self.handle = h.value
        self._tasks = set()

    def task_create(self, in_size: int, out_size: int) -> Task:
        h = _vp()
        st = load().crystal_task_create(self.handle, in_size, out_size, ctypes.byref(h))
        if st != CRYSTAL_OK:
            raise CrystalError(st, "crystal_task_create")
        t = Task(self, h.value, in_size, out_size)
        self._tasks.add(t)
        return t

    @staticmethod
    def task_array(tasks: Sequence[Task]):
        """The job handles as a C array, for the *_many calls (build it once
        for a set of jobs submitted again and again)."""
        return (_vp * len(tasks))(*[t.handle for t in tasks])

    def submit_many(self, tasks, kind: int, p: Optional[crystal_hash_params] = None,
                    callback=None, user=None) -> int:
        """crystal_task_submit_many: all of ``tasks`` (Task list or
        :meth:`task_array`) or none."""
        arr = tasks if isinstance(tasks, ctypes.Array) else self.task_array(tasks)
        cb = callback if callback is not None else crystal_callback()
        self._cb_keepalive = cb
        return load().crystal_task_submit_many(arr, len(arr), kind, ctypes.byref(p) if p is not None else None,
                                               cb, user)

    def wait_many(self, tasks, timeout_ns: int = -1) -> int:
        """crystal_task_wait_many: every job of ``tasks`` finished (first
        non-OK status in order), or CRYSTAL_ETIMEDOUT."""
        arr = tasks if isinstance(tasks, ctypes.Array) else self.task_array(tasks)
        return load().crystal_task_wait_many(arr, len(arr), timeout_ns)

    def timing_many(self, tasks) -> np.ndarray:
        """crystal_task_timing_many: (n, 3) uint64 stamps (submit, dispatch,
        done) of ``tasks``."""
        arr = tasks if isinstance(tasks, ctypes.Array) else self.task_array(tasks)
        out = np.zeros((len(arr), 3), dtype=np.uint64)
        check(load().crystal_task_timing_many(arr, len(arr), out.ctypes.data), "crystal_task_timing_many")
        return out

    def serve(self, source: np.ndarray, requests: np.ndarray, direct: Optional[crystal_hash_params] = None,
              sliding: Optional[crystal_hash_params] = None, capture: Optional[np.ndarray] = None,
              copy_threads: int = 4, source_pinned: bool = False, arrival_order: bool = False,
              bypass_ns: int = 0, ring_bytes: int = 0, ring_max_request: int = 0):
        """crystal_serve: play ``requests`` (REQUEST_DTYPE, arrival order)
        against this context.  ``arrival_order`` admits strictly in arrival
        order; otherwise later requests that fit may pass a blocked oldest one
        for ``bypass_ns`` (0: the library's default).  ``ring_bytes`` > 0
        stages requests of at most ``ring_max_request`` bytes (0: the
        library's default) through an input ring so that their copies merge.
        Returns (status, results, wall_ns)."""
        src = np.ascontiguousarray(source, dtype=np.uint8)
        req = np.ascontiguousarray(requests, dtype=REQUEST_DTYPE)
        res = np.zeros(len(req), dtype=RESULT_DTYPE)
        cfg = crystal_serve_config()
        cfg.copy_threads = copy_threads
        cfg.flags = (CRYSTAL_SERVE_SOURCE_PINNED if source_pinned else 0) | \
            (CRYSTAL_SERVE_ARRIVAL_ORDER if arrival_order else 0)
        cfg.bypass_ns = bypass_ns
        cfg.ring_bytes, cfg.ring_max_request = ring_bytes, ring_max_request
        cfg.direct_params = ctypes.cast(ctypes.pointer(direct), ctypes.c_void_p) if direct is not None else None
        cfg.sliding_params = ctypes.cast(ctypes.pointer(sliding), ctypes.c_void_p) if sliding is not None else None
        if capture is not None:
            cfg.capture, cfg.capture_bytes = capture.ctypes.data, capture.nbytes
        wall = _u64()
        st = load().crystal_serve(self.handle, src.ctypes.data, src.nbytes, req.ctypes.data, len(req),
                                  ctypes.byref(cfg), res.ctypes.data, ctypes.byref(wall))
        return st, res, wall.value

    def stream_staged(self, units: Sequence[np.ndarray], kind: int, out_size: int,
                      p: Optional[crystal_hash_params] = None, copy_threads: int = 4, ring_jobs: int = 0,
                      out_stride: Optional[int] = None, keep_outputs: bool = True):
        """crystal_stream_staged: hash ``units`` (host uint8 arrays, e.g. views
        of one pageable buffer) through a ring of pinned jobs filled by
        ``copy_threads`` C++ threads.  Returns (status, results, wall_ns,
        outputs) with ``outputs`` an (n, out_stride) uint8 array or None."""
        n = len(units)
        arrs = [np.ascontiguousarray(u, dtype=np.uint8) for u in units]
        ptrs = (_vp * max(n, 1))(*[a.ctypes.data for a in arrs])
        sizes = np.array([a.nbytes for a in arrs], dtype=np.uint64)
        stride = out_stride if out_stride is not None else out_size
        outs = np.zeros((n, stride), dtype=np.uint8) if keep_outputs and n else None
        res = np.zeros(n, dtype=RESULT_DTYPE)
        cfg = crystal_stream_config()
        cfg.kind, cfg.copy_threads, cfg.ring_jobs, cfg.reserved, cfg.out_size = kind, copy_threads, ring_jobs, 0, \
            out_size
        cfg.params = ctypes.cast(ctypes.pointer(p), ctypes.c_void_p) if p is not None else None
        wall = _u64()
        st = load().crystal_stream_staged(self.handle, ptrs, sizes.ctypes.data, n, ctypes.byref(cfg),
                                          outs.ctypes.data if outs is not None else None, stride,
                                          res.ctypes.data, ctypes.byref(wall))
        del arrs
        return st, res, wall.value, outs

    def set_geometry(self, size_class: int, g: Optional[crystal_geometry]) -> None:
        """crystal_set_geometry (size_class -1: every class; g None: defaults)."""
        check(load().crystal_set_geometry(self.handle, size_class, ctypes.byref(g) if g is not None else None),
              "crystal_set_geometry")

    def get_geometry(self, size_class: int) -> crystal_geometry:
        g = crystal_geometry()
        check(load().crystal_get_geometry(self.handle, size_class, ctypes.byref(g)), "crystal_get_geometry")
        return g

    def config(self) -> crystal_config:
        c = crystal_config()
        check(load().crystal_get_config(self.handle, ctypes.byref(c)), "crystal_get_config")
        return c

    def prepare_graphs(self) -> None:
        """crystal_prepare_graphs: capture every stream slot's batch graphs
        now (the context must be idle)."""
        check(load().crystal_prepare_graphs(self.handle), "crystal_prepare_graphs")

    def stats(self) -> crystal_stats:
        s = crystal_stats()
        check(load().crystal_get_stats(self.handle, ctypes.byref(s)), "crystal_get_stats")
        return s

    def shutdown(self) -> int:
        if self.handle is None:
            return CRYSTAL_OK
        st = load().crystal_shutdown(self.handle)
        self.handle = None
        self._tasks.clear()
        return st

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.shutdown()


class CrystalError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {load().crystal_strerror(status).decode()} ({status})")


# ---- stateless batch launchers on torch-owned device memory ---------------------

def _align(x: int, a: int) -> int:
    return (x + a - 1) // a * a


class DeviceBatch:
    """A batch of units living in one device input buffer (a torch uint8
    tensor), with outputs, scratch and the descriptor in torch-owned device
    memory.  ``offsets``/``sizes`` locate each unit in ``d_input``; units are
    reordered direct-first as the descriptor requires, and results come back
    in the caller's order.  ``out_misalign`` (multiples of 4, cycled over the
    units) places each output that many bytes past a 256-byte boundary; the
    C ABI only asks for 4-byte aligned outputs."""

    def __init__(self, d_input, offsets: Sequence[int], sizes: Sequence[int], kinds: Sequence[int],
                 p: Optional[crystal_hash_params] = None, out_sizes: Optional[Sequence[int]] = None,
                 per_unit_params: Optional[Sequence[crystal_hash_params]] = None,
                 out_misalign: Optional[Sequence[int]] = None):
        import torch

        L = load()
        if not d_input.is_cuda or d_input.dtype != torch.uint8:
            raise ValueError("d_input must be a CUDA uint8 tensor")
        n_units = len(sizes)
        self.device = d_input.device
        self.kinds = list(kinds)
        self.sizes = [int(s) for s in sizes]
        order = [i for i in range(n_units) if kinds[i] in DIRECT_KINDS] + \
                [i for i in range(n_units) if kinds[i] in SLIDING_KINDS]
        if len(order) != n_units:
            raise ValueError("kinds must be direct or sliding")
        self.order = order
        self.n_direct = sum(1 for k in kinds if k in DIRECT_KINDS)
        self.n_sliding = n_units - self.n_direct
        plist = per_unit_params or [p if p is not None else params()] * n_units
        self.params = plist
        # output and scratch layout, 256-byte aligned per unit
        self.out_off, self.out_size, self.scr_off = [0] * n_units, [0] * n_units, [0] * n_units
        o = s = 0
        for i in range(n_units):
            pi = plist[i]
            if out_sizes is not None:
                osz = int(out_sizes[i])
            elif kinds[i] in DIRECT_KINDS:
                osz = digest_size(kinds[i])
            else:
                osz = L.crystal_out_bytes(kinds[i], self.sizes[i], ctypes.byref(pi))
            mis = int(out_misalign[i % len(out_misalign)]) if out_misalign else 0
            if mis % 4:
                raise ValueError("outputs must stay 4-byte aligned")
            self.out_off[i], self.out_size[i] = o + mis, osz
            o = _align(o + mis + osz, 256)
            sb = L.crystal_scratch_bytes(kinds[i], self.sizes[i], osz, ctypes.byref(pi))
            self.scr_off[i] = s
            s = _align(s + max(sb, 16), 256)
        self.d_out = torch.zeros(max(o, 256), dtype=torch.uint8, device=self.device)
        self.d_scratch = torch.zeros(max(s, 256), dtype=torch.uint8, device=self.device)
        self.d_input = d_input
        nbytes = int(L.crystal_batch_bytes(n_units))
        host = np.zeros(nbytes, dtype=np.uint8)
        units = host[BATCH_HEADER_BYTES:].view(UNIT_DTYPE)
        base_in, base_out, base_scr = d_input.data_ptr(), self.d_out.data_ptr(), self.d_scratch.data_ptr()
        for k, i in enumerate(order):
            pi = plist[i]
            u = units[k]
            u["in"] = base_in + int(offsets[i])
            u["n"] = self.sizes[i]
            u["out"] = base_out + self.out_off[i]
            u["scratch"] = base_scr + self.scr_off[i]
            u["out_cap"] = self.out_size[i]
            direct = kinds[i] in DIRECT_KINDS
            u["seg_bytes"] = (pi.segment_bytes if direct else pi.chunk_segment_bytes) or 4096
            u["window"] = pi.window_bytes or 20
            u["mask"], u["target"], u["kind"] = pi.mask, pi.target, kinds[i]
        st = L.crystal_batch_plan(host.ctypes.data, self.n_direct, self.n_sliding)
        check(st, "crystal_batch_plan")
        self.host_desc = host
        self.d_desc = torch.from_numpy(host).to(self.device)
        self.total_segments = int(host[8:16].view("<u8")[0])
        self.total_tiles = int(host[16:24].view("<u8")[0])

    @staticmethod
    def _stream(stream) -> int:
        import torch

        s = stream if stream is not None else torch.cuda.current_stream()
        return s.cuda_stream

    def _launch(self, fn: str, stream=None) -> None:
        st = getattr(load(), fn)(self.d_desc.data_ptr(), self._stream(stream))
        check(st, fn)

    def launch(self, stream=None):
        self._launch("crystal_launch_batch", stream)

    def launch_direct(self, stream=None):
        self._launch("crystal_launch_direct", stream)

    def launch_direct_segments(self, stream=None):
        self._launch("crystal_launch_direct_segments", stream)

    def launch_direct_outer(self, stream=None):
        self._launch("crystal_launch_direct_outer", stream)

    def launch_sliding(self, stream=None):
        self._launch("crystal_launch_sliding", stream)

    def launch_sliding_windows(self, stream=None):
        self._launch("crystal_launch_sliding_windows", stream)

    def launch_sliding_chunks(self, stream=None):
        self._launch("crystal_launch_sliding_chunks", stream)

    def launch_sliding_digests(self, stream=None):
        self._launch("crystal_launch_sliding_digests", stream)

    def device_status(self) -> int:
        return int(self.d_desc[:64].cpu().numpy()[28:32].view("<u4")[0])

    def outputs(self) -> List[bytes]:
        """Each unit's output bytes, in the caller's order."""
        host = self.d_out.cpu().numpy()
        return [host[self.out_off[i]:self.out_off[i] + self.out_size[i]].tobytes() for i in range(len(self.sizes))]


def alu_probe(kind: int, ctas_per_sm: int, iters: int, sink, stream=None) -> int:
    """Launch crystal_alu_probe on ``stream`` (a torch stream; default: the
    current one); ``sink`` is a CUDA tensor of at least 4 bytes.  Returns the
    work of the launch (windows or instructions)."""
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    w = _u64()
    check(load().crystal_alu_probe(kind, ctas_per_sm, iters, 0x9E3779B9, sink.data_ptr(), s.cuda_stream,
                                   ctypes.byref(w)), "crystal_alu_probe")
    return int(w.value)
