"""Multi-threaded CPU compaction (cpu_mt.c), timed by the benchmark for
context beside the oracle. Not the oracle, and not used by the product: test
and benchmark infrastructure, like the rest of this package."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpu_mt.c")
_SO = os.path.join(_HERE, "_build", "libka_cpu_mt.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile cpu_mt.c with gcc -O2 -pthread."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-pthread", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.cpu_mt_compact_lt.restype = ctypes.c_uint64
            L.cpu_mt_compact_lt.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p,
                                            ctypes.c_int]
            _lib = L
    return _lib


def compact_lt(x: np.ndarray, t: int, threads: int):
    """(kept entries, count) of x < t, with `threads` threads."""
    x = np.ascontiguousarray(x, dtype=np.uint32)
    y = np.empty(max(x.size, 1), dtype=np.uint32)
    k = int(lib().cpu_mt_compact_lt(x.ctypes.data, x.size, t, y.ctypes.data, threads))
    if k == 2**64 - 1:
        raise RuntimeError("threads could not be started")
    return y[:k], k
