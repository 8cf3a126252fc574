"""CPU oracle for the compaction pipelines (test infrastructure).

Only the tests, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg
may import this package. The product library never does, and this package never
imports the product: the two share no code. The arithmetic lives in
`ka_oracle.c` (plain sequential C, compiled -O2 with gcc); this wrapper only
builds it, passes numpy arrays to it, and composes the per-stage definitions
into the pipelines the paper describes:

  * single compaction (Sec. 4.1): keep-predicate, stable order, new length;
  * flag / exclusive-scan / move phases (Sec. 4.1, Listing 5);
  * composed pipeline C = B o A, i.e. C(msg) = B(A(msg)) (Sec. 3.5), with the
    output of one stage and its length feeding the next;
  * fuseFillsLiterals = move o count o prepare (Sec. 4.1, Listing 5).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ka_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libka_oracle.so")

# The oracle's own predicate numbering (see ka_oracle.c).
PRED_IDS = {"and_mask_eq0": 0, "lt": 1, "topbits_lt": 2, "popc_odd": 3, "mod_ne0": 4, "ne": 5, "all": 6}

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ka_oracle.c into a shared library with gcc -O2 (no CUDA)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def bind(L):
    """Declare the C signatures on a loaded oracle library and return it."""
    u32p = ctypes.POINTER(ctypes.c_uint32)
    L.ora_splitmix64.restype = ctypes.c_uint64
    L.ora_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    L.ora_generate.restype = None
    L.ora_generate.argtypes = [ctypes.c_uint64, ctypes.c_uint64, u32p]
    L.ora_keep.restype = ctypes.c_int
    L.ora_keep.argtypes = [ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32]
    L.ora_predicate_map.restype = ctypes.c_int
    L.ora_predicate_map.argtypes = [u32p, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32, u32p]
    L.ora_exclusive_scan.restype = ctypes.c_uint32
    L.ora_exclusive_scan.argtypes = [u32p, ctypes.c_uint64, u32p]
    L.ora_scatter.restype = None
    L.ora_scatter.argtypes = [u32p, u32p, u32p, ctypes.c_uint64, u32p]
    L.ora_compact.restype = ctypes.c_uint64
    L.ora_compact.argtypes = [u32p, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32, u32p]
    L.ora_map_hash.restype = None
    L.ora_map_hash.argtypes = [u32p, ctypes.c_uint64, u32p]
    L.ora_prepare_index.restype = None
    L.ora_prepare_index.argtypes = [u32p, u32p, ctypes.c_uint64, u32p]
    L.ora_mandelbrot.restype = None
    L.ora_mandelbrot.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                 ctypes.c_float, ctypes.c_uint32, u32p]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = bind(ctypes.CDLL(build()))
    return _lib


def use_library(L):
    """Swap the loaded oracle library (tests that plant a mistake in a copy of
    ka_oracle.c use this to check that the pins catch it). Returns the old one."""
    global _lib
    with _lock:
        old, _lib = _lib, L
    return old


def _p(a: np.ndarray):
    assert a.dtype == np.uint32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _u32(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.uint32)


def pred_id(name: str) -> int:
    return PRED_IDS[name]


# ----------------------------------------------------------------------------
# Single functions (one C call each).
# ----------------------------------------------------------------------------

def splitmix64(seed: int, i: int) -> int:
    return int(lib().ora_splitmix64(seed & (2**64 - 1), i))


def generate(seed: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint32)
    if n:
        lib().ora_generate(seed & (2**64 - 1), n, _p(out))
    return out


def keep(pred: str, param: int, x: int) -> int:
    return int(lib().ora_keep(pred_id(pred), param, x))


def predicate_map(x, pred: str, param: int) -> np.ndarray:
    x = _u32(x)
    f = np.empty(x.size, dtype=np.uint32)
    if x.size and lib().ora_predicate_map(_p(x), x.size, pred_id(pred), param, _p(f)) != 0:
        raise ValueError("bad predicate %s(%d)" % (pred, param))
    return f


def exclusive_scan(v):
    """Returns (o, total)."""
    v = _u32(v)
    o = np.empty(v.size, dtype=np.uint32)
    total = int(lib().ora_exclusive_scan(_p(v), v.size, _p(o))) if v.size else 0
    return o, total


def scatter(x, f, o, out_len: int) -> np.ndarray:
    x, f, o = _u32(x), _u32(f), _u32(o)
    y = np.zeros(out_len, dtype=np.uint32)
    if x.size:
        lib().ora_scatter(_p(x), _p(f), _p(o), x.size, _p(y))
    return y


def compact(x, pred: str, param: int):
    """Returns (y, k): the kept entries of x in order and their number."""
    x = _u32(x)
    y = np.empty(x.size, dtype=np.uint32)
    k = int(lib().ora_compact(_p(x), x.size, pred_id(pred), param, _p(y))) if x.size else 0
    if k == 2**64 - 1:
        raise ValueError("bad predicate %s(%d)" % (pred, param))
    return y[:k].copy(), k


def map_hash(x) -> np.ndarray:
    x = _u32(x)
    h = np.empty(x.size, dtype=np.uint32)
    if x.size:
        lib().ora_map_hash(_p(x), x.size, _p(h))
    return h


def prepare_index(chunk_ids, literals) -> np.ndarray:
    a, b = _u32(chunk_ids), _u32(literals)
    assert a.size == b.size
    out = np.empty(2 * a.size, dtype=np.uint32)
    if a.size:
        lib().ora_prepare_index(_p(a), _p(b), a.size, _p(out))
    return out


# ----------------------------------------------------------------------------
# Compositions (Sec. 3.5: C = B o A feeds A's result, with its length, to B).
# ----------------------------------------------------------------------------

def mandelbrot(width: int, height: int, re_min: float, im_min: float, re_max: float, im_max: float,
               max_iter: int) -> np.ndarray:
    """Escape-time image (Sec. 5.4), uint32 [height, width], row 0 at im_min."""
    out = np.zeros(width * height, dtype=np.uint32)
    lib().ora_mandelbrot(width, height, re_min, im_min, re_max, im_max, max_iter, _p(out))
    return out.reshape(height, width)


# The rectangle of the paper's Mandelbrot workload (Sec. 5.4): from
# -0.5 - 0.7375i to 0.1 - 0.1375i.
MANDELBROT_REGION = (-0.5, -0.7375, 0.1, -0.1375)


def three_phase(x, pred: str, param: int):
    """Flag, exclusive scan, move (Sec. 4.1). Returns (f, o, total, y)."""
    f = predicate_map(x, pred, param)
    o, total = exclusive_scan(f)
    y = scatter(x, f, o, total)
    return f, o, total, y


def run_stage(x, stage):
    """One pipeline stage on the live array x; stage has .kind/.pred/.param."""
    if stage.kind == "map_hash":
        return map_hash(x)
    if stage.kind == "compact":
        y, _ = compact(x, stage.pred, stage.param)
        return y
    raise ValueError(stage.kind)


def pipeline(x, stages):
    """Composition of stages, first stage first. Returns the per-stage outputs."""
    outs = []
    cur = _u32(x)
    for st in stages:
        cur = run_stage(cur, st)
        outs.append(cur)
    return outs


def fuse_fills_literals(chunk_ids, literals):
    """move o count o prepare: interleave, then remove zero entries (Sec. 4.1)."""
    index = prepare_index(chunk_ids, literals)
    return compact(index, "ne", 0)
