"""B300-native CrystalGPU hashing pipeline.

A stream of host data units hashed on one GPU -- MD5 direct hashing and MD5
sliding-window (content-defined chunking) hashing -- behind the job runtime of
the CrystalGPU paper: a pooled device/pinned-host buffer arena, copy/compute
overlap across streams, and a master thread that batches, dispatches, polls
and calls back.  The compute path is ``libcrystal.so`` (CUDA for sm_103a plus
a C++ runtime); :mod:`.crystal` is its ctypes binding and :mod:`.inputs` the
seeded synthetic workload generators.
"""
from . import crystal, inputs  # noqa: F401

__all__ = ["crystal", "inputs"]
