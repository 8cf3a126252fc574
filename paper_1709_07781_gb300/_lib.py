"""ctypes binding of libka.so: the C entry points of include/ka.h under the same
names. Argument marshalling only: device pointers may be given as ints or as
torch tensors (their data_ptr), streams as ints, torch streams, or None; every
computation happens in the library's CUDA kernels.

Calls return the C status code (0 = KA_OK); calls with C out-parameters return
(status, value...). `check(status)` raises KaError for a non-zero status.
The library must have been built (build.py, or __graft_entry__.build()); a
missing library raises at import, and there is no other code path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libka.so")

c_u32p = ctypes.POINTER(ctypes.c_uint32)
c_vp = ctypes.c_void_p

STATUS = {
    0: "KA_OK", -1: "KA_E_ARG", -2: "KA_E_TYPE", -3: "KA_E_OOM", -4: "KA_E_BUDGET", -5: "KA_E_STALE",
    -6: "KA_E_CUDA", -7: "KA_E_DEVICE_TIMEOUT", -8: "KA_E_CLOSED", -9: "KA_E_NOT_SERIALIZABLE",
    -10: "KA_E_TIMEOUT", -11: "KA_E_UNSUPPORTED", -12: "KA_E_INJECTED", -13: "KA_E_WORKSPACE",
    -14: "KA_E_TOO_LARGE",
}
globals().update({v: k for k, v in STATUS.items()})

PRED = {"and_mask_eq0": 0, "lt": 1, "topbits_lt": 2, "popc_odd": 3, "mod_ne0": 4, "ne": 5, "all": 6}
KA_PRED_AND_MASK_EQ0, KA_PRED_LT, KA_PRED_TOPBITS_LT, KA_PRED_POPC_ODD, KA_PRED_MOD_NE0, KA_PRED_NE, KA_PRED_ALL = range(7)
KA_XFORM_NONE, KA_XFORM_HASH = 0, 1
KA_KERNEL_COMPACT, KA_KERNEL_SCAN, KA_KERNEL_BATCH = 0, 1, 2
(KA_STAGE_GENERATE, KA_STAGE_MAP_HASH, KA_STAGE_PREDICATE, KA_STAGE_EXSCAN, KA_STAGE_SCATTER,
 KA_STAGE_COMPACT, KA_STAGE_PREPARE, KA_STAGE_EMPTY, KA_STAGE_MANDELBROT) = range(9)
KA_U32 = 0
KA_READ, KA_WRITE, KA_READ_WRITE = 1, 2, 3
KA_MSG_MAX_REFS = 4


class KaError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__("%s (%d)%s" % (STATUS.get(status, "?"), status, (": " + what) if what else ""))


def check(status, what: str = ""):
    s = status[0] if isinstance(status, tuple) else status
    if s != 0:
        raise KaError(s, what)
    return status


class ka_tile(ctypes.Structure):
    _fields_ = [("block", ctypes.c_uint32), ("ipt", ctypes.c_uint32)]


class ka_batch_item(ctypes.Structure):
    _fields_ = [("in_", c_vp), ("out", c_vp), ("n_ptr", c_vp), ("count", c_vp), ("n", ctypes.c_uint32),
                ("pred", ctypes.c_int32), ("param", ctypes.c_uint32), ("xform", ctypes.c_uint32)]


class ka_gen_item(ctypes.Structure):
    _fields_ = [("out", c_vp), ("seed", ctypes.c_uint64), ("n", ctypes.c_uint32), ("pad", ctypes.c_uint32)]


class ka_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("debug", ctypes.c_int32), ("stream", c_vp),
                ("budget_bytes", ctypes.c_uint64), ("autotune_cache", ctypes.c_char_p)]


class ka_stage_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("pred", ctypes.c_int32), ("param", ctypes.c_uint32),
                ("xform", ctypes.c_uint32), ("tile", ka_tile)]


class ka_msg(ctypes.Structure):
    _fields_ = [("n_refs", ctypes.c_uint32), ("refs", c_vp * KA_MSG_MAX_REFS), ("h_in", c_u32p),
                ("h_n", ctypes.c_uint64), ("h_out", c_u32p), ("h_out_cap", ctypes.c_uint64),
                ("seed", ctypes.c_uint64), ("gen_n", ctypes.c_uint64), ("count", ctypes.c_uint64),
                ("status", ctypes.c_int32)]


class ka_serve_stage(ctypes.Structure):
    _fields_ = [("pred", ctypes.c_int32), ("param", ctypes.c_uint32), ("xform", ctypes.c_uint32)]


class ka_serve_request(ctypes.Structure):
    _fields_ = [("arrival_s", ctypes.c_double), ("seed", ctypes.c_uint64), ("n", ctypes.c_uint32),
                ("n_stages", ctypes.c_uint32), ("stages", ka_serve_stage * 4), ("h_out", c_u32p),
                ("h_out_cap", ctypes.c_uint64)]


class ka_serve_result(ctypes.Structure):
    _fields_ = [("admit_s", ctypes.c_double), ("done_s", ctypes.c_double), ("count", ctypes.c_uint32),
                ("status", ctypes.c_int32)]


class ka_serve_options(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_uint32), ("max_inflight", ctypes.c_uint32), ("budget_bytes", ctypes.c_uint64),
                ("time_scale", ctypes.c_double), ("tile", ka_tile), ("flags", ctypes.c_uint32)]


class ka_serve_stats(ctypes.Structure):
    _fields_ = [("wall_s", ctypes.c_double), ("elements", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("iterations", ctypes.c_uint64), ("peak_bytes", ctypes.c_uint64),
                ("max_inflight_seen", ctypes.c_uint32), ("rejected", ctypes.c_uint32),
                ("graph_launches", ctypes.c_uint64), ("lone_ticks", ctypes.c_uint64),
                ("max_step_s", ctypes.c_double), ("slow_steps", ctypes.c_uint64),
                ("max_alloc_s", ctypes.c_double), ("max_free_s", ctypes.c_double),
                ("max_issue_s", ctypes.c_double), ("max_poll_s", ctypes.c_double)]


MONITOR_FN = ctypes.CFUNCTYPE(None, c_vp, ctypes.c_int32)

# name -> (restype, argtypes)
_SIGS = {
    "ka_strerror": (ctypes.c_char_p, [ctypes.c_int32]),
    "ka_version": (ctypes.c_int32, []),
    "ka_last_cuda_error": (ctypes.c_int32, []),
    "ka_workspace_size": (ctypes.c_int32, [ctypes.c_uint64, ctypes.POINTER(ka_tile), ctypes.POINTER(ctypes.c_uint64)]),
    "ka_workspace_init": (ctypes.c_int32, [c_vp, ctypes.c_uint64, c_vp]),
    "ka_workspace_status": (ctypes.c_int32, [c_vp, c_vp, ctypes.POINTER(ctypes.c_int32)]),
    "ka_workspace_set_spin_limit": (ctypes.c_int32, [c_vp, ctypes.c_uint32, c_vp]),
    "ka_generate": (ctypes.c_int32, [c_vp, ctypes.c_uint64, ctypes.c_uint64, c_vp]),
    "ka_map_hash": (ctypes.c_int32, [c_vp, ctypes.c_uint64, c_vp, c_vp, c_vp, c_vp]),
    "ka_predicate": (ctypes.c_int32, [c_vp, ctypes.c_uint64, c_vp, ctypes.c_int32, ctypes.c_uint32, c_vp, c_vp]),
    "ka_exclusive_scan": (ctypes.c_int32, [c_vp, ctypes.c_uint64, c_vp, c_vp, c_vp, c_vp, ctypes.c_uint64,
                                           ctypes.POINTER(ka_tile), c_vp]),
    "ka_scatter": (ctypes.c_int32, [c_vp, c_vp, c_vp, ctypes.c_uint64, c_vp, c_vp, c_vp]),
    "ka_compact": (ctypes.c_int32, [c_vp, ctypes.c_uint64, c_vp, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint32,
                                    c_vp, c_vp, c_vp, ctypes.c_uint64, ctypes.POINTER(ka_tile), c_vp]),
    "ka_compact_static": (ctypes.c_int32, [c_vp, ctypes.c_uint64, c_vp, ctypes.c_int32, ctypes.c_uint32,
                                           ctypes.c_uint32, c_vp, c_vp, ctypes.POINTER(ka_tile), c_vp]),
    "ka_compact_static_workspace": (ctypes.c_int32, [c_vp, ctypes.POINTER(c_vp), ctypes.POINTER(ctypes.c_uint64)]),
    "ka_three_phase_workspace_size": (ctypes.c_int32, [ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]),
    "ka_compact_three_phase": (ctypes.c_int32, [c_vp, ctypes.c_uint64, c_vp, ctypes.c_int32, ctypes.c_uint32,
                                                ctypes.c_uint32, c_vp, c_vp, c_vp, ctypes.c_uint64, c_vp]),
    "ka_compact_host_scratch_size": (ctypes.c_int32, [ctypes.c_uint64, ctypes.c_uint32,
                                                      ctypes.POINTER(ctypes.c_uint64)]),
    "ka_compact_host": (ctypes.c_int32, [c_vp, ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                         ctypes.POINTER(c_vp), ctypes.POINTER(ctypes.c_uint64), ctypes.c_uint64,
                                         c_vp, ctypes.c_uint64]),
    "ka_mandelbrot": (ctypes.c_int32, [c_vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_float, ctypes.c_float,
                                       ctypes.c_float, ctypes.c_float, ctypes.c_uint32, c_vp]),
    "ka_prepare_index": (ctypes.c_int32, [c_vp, c_vp, ctypes.c_uint64, c_vp, c_vp, c_vp, c_vp]),
    "ka_batch_workspace_size": (ctypes.c_int32, [ctypes.c_uint32, ctypes.c_uint64, ctypes.POINTER(ka_tile),
                                                 ctypes.POINTER(ctypes.c_uint64)]),
    "ka_compact_batch": (ctypes.c_int32, [c_vp, ctypes.c_uint32, ctypes.c_uint32, c_vp, ctypes.c_uint64,
                                          ctypes.POINTER(ka_tile), ctypes.c_uint32, c_vp]),
    "ka_generate_batch": (ctypes.c_int32, [c_vp, ctypes.c_uint32, ctypes.c_uint32, c_vp, ctypes.c_uint64, c_vp]),
    "ka_autotune": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_uint64, ctypes.c_char_p, ctypes.POINTER(ka_tile),
                                     ctypes.POINTER(ctypes.c_float), c_vp]),
    "ka_tile_for": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_uint64, ctypes.POINTER(ka_tile)]),
    "ka_autotune_load": (ctypes.c_int32, [ctypes.c_char_p]),
    "ka_system_create": (ctypes.c_int32, [ctypes.POINTER(ka_config), ctypes.POINTER(c_vp)]),
    "ka_system_destroy": (ctypes.c_int32, [c_vp, ctypes.c_int32]),
    "ka_system_pool_bytes": (ctypes.c_int32, [c_vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "ka_ref_wrap": (ctypes.c_int32, [c_vp, c_vp, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.POINTER(c_vp)]),
    "ka_ref_alloc": (ctypes.c_int32, [c_vp, ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(c_vp)]),
    "ka_ref_count": (ctypes.c_int32, [c_vp, ctypes.POINTER(ctypes.c_uint64)]),
    "ka_ref_info": (ctypes.c_int32, [c_vp, ctypes.POINTER(c_vp), ctypes.POINTER(ctypes.c_uint64),
                                     ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "ka_ref_retain": (ctypes.c_int32, [c_vp]),
    "ka_ref_release": (ctypes.c_int32, [c_vp]),
    "ka_ref_serialize": (ctypes.c_int32, [c_vp, c_vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]),
    "ka_spawn_stage": (ctypes.c_int32, [c_vp, ctypes.POINTER(ka_stage_desc), ctypes.POINTER(c_vp)]),
    "ka_compose": (ctypes.c_int32, [c_vp, c_vp, ctypes.POINTER(c_vp)]),
    "ka_actor_arity": (ctypes.c_int32, [c_vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "ka_actor_release": (ctypes.c_int32, [c_vp]),
    "ka_request": (ctypes.c_int32, [c_vp, ctypes.POINTER(ka_msg), ctypes.POINTER(c_vp)]),
    "ka_receive": (ctypes.c_int32, [c_vp, ctypes.c_int64, ctypes.POINTER(ka_msg)]),
    "ka_debug_device_cache": (ctypes.c_int32, [ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                               ctypes.c_uint32, ctypes.POINTER(ctypes.c_int32)]),
    "ka_debug_pred_keep": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint32,
                                            ctypes.POINTER(ctypes.c_int32)]),
    "ka_debug_fail_stage": (ctypes.c_int32, [c_vp, ctypes.c_int32]),
    "ka_debug_kill_dispatcher": (ctypes.c_int32, [c_vp]),
    "ka_system_monitor": (ctypes.c_int32, [c_vp, MONITOR_FN, c_vp]),
    "ka_bench_request_loop": (ctypes.c_int32, [c_vp, ctypes.POINTER(ka_msg), ctypes.c_uint32, ctypes.c_uint32,
                                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64)]),
    "ka_bench_direct_chain": (ctypes.c_int32, [ctypes.POINTER(ka_stage_desc), ctypes.c_uint32, c_vp, ctypes.c_uint64,
                                               ctypes.c_uint32, c_vp, ctypes.c_uint32, ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_uint64)]),
    "ka_serve_run": (ctypes.c_int32, [c_vp, ctypes.POINTER(ka_serve_request), ctypes.c_uint32,
                                      ctypes.POINTER(ka_serve_options), ctypes.POINTER(ka_serve_result),
                                      ctypes.POINTER(ka_serve_stats)]),
}

if not os.path.exists(LIB_PATH):
    raise ImportError("libka.so is not built (%s); run __graft_entry__.build() or "
                      "python paper_1709_07781_gb300/build.py" % LIB_PATH)

lib = ctypes.CDLL(LIB_PATH)
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args

DECLARED = tuple(_SIGS)


def ptr(x):
    """Device/host pointer of an int, a torch tensor, a numpy array, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError("not a pointer: %r" % type(x))


def stream_ptr(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _tile(t):
    if t is None:
        return None
    if isinstance(t, ka_tile):
        return ctypes.byref(t)
    return ctypes.byref(ka_tile(int(t[0]), int(t[1])))


def ka_strerror(status: int) -> str:
    return lib.ka_strerror(status).decode()


def ka_version() -> int:
    return lib.ka_version()


def ka_last_cuda_error() -> int:
    return lib.ka_last_cuda_error()


def ka_workspace_size(capacity: int, tile=None):
    out = ctypes.c_uint64(0)
    s = lib.ka_workspace_size(capacity, _tile(tile), ctypes.byref(out))
    return s, out.value


def ka_workspace_init(d_ws, nbytes: int, stream=None) -> int:
    return lib.ka_workspace_init(ptr(d_ws), nbytes, stream_ptr(stream))


def ka_workspace_status(d_ws, stream=None):
    out = ctypes.c_int32(0)
    s = lib.ka_workspace_status(ptr(d_ws), stream_ptr(stream), ctypes.byref(out))
    return s, out.value


def ka_workspace_set_spin_limit(d_ws, polls: int, stream=None) -> int:
    return lib.ka_workspace_set_spin_limit(ptr(d_ws), polls, stream_ptr(stream))


def ka_generate(d_out, n: int, seed: int, stream=None) -> int:
    return lib.ka_generate(ptr(d_out), n, seed & (2**64 - 1), stream_ptr(stream))


def ka_map_hash(d_in, n: int, d_n, d_out, d_n_out=None, stream=None) -> int:
    return lib.ka_map_hash(ptr(d_in), n, ptr(d_n), ptr(d_out), ptr(d_n_out), stream_ptr(stream))


def ka_predicate(d_x, n: int, d_n, pred: int, param: int, d_flags, stream=None) -> int:
    return lib.ka_predicate(ptr(d_x), n, ptr(d_n), pred, param, ptr(d_flags), stream_ptr(stream))


def ka_exclusive_scan(d_in, n: int, d_n, d_out, d_total, d_ws, ws_bytes: int, tile=None, stream=None) -> int:
    return lib.ka_exclusive_scan(ptr(d_in), n, ptr(d_n), ptr(d_out), ptr(d_total), ptr(d_ws), ws_bytes,
                                 _tile(tile), stream_ptr(stream))


def ka_scatter(d_x, d_flags, d_offsets, n: int, d_n, d_out, stream=None) -> int:
    return lib.ka_scatter(ptr(d_x), ptr(d_flags), ptr(d_offsets), n, ptr(d_n), ptr(d_out), stream_ptr(stream))


def ka_compact(d_in, n: int, d_n, pred: int, param: int, xform: int, d_out, d_count, d_ws, ws_bytes: int,
               tile=None, stream=None) -> int:
    return lib.ka_compact(ptr(d_in), n, ptr(d_n), pred, param, xform, ptr(d_out), ptr(d_count), ptr(d_ws),
                          ws_bytes, _tile(tile), stream_ptr(stream))


KA_STATIC_MAX_N = 1 << 24


def ka_compact_static(d_in, n: int, d_n, pred: int, param: int, xform: int, d_out, d_count, tile=None,
                      stream=None) -> int:
    return lib.ka_compact_static(ptr(d_in), n, ptr(d_n), pred, param, xform, ptr(d_out), ptr(d_count),
                                 _tile(tile), stream_ptr(stream))


def ka_compact_static_workspace(stream=None):
    """(status, device address, bytes) of the current device's shared array."""
    p, nb = c_vp(0), ctypes.c_uint64(0)
    s = lib.ka_compact_static_workspace(stream_ptr(stream), ctypes.byref(p), ctypes.byref(nb))
    return s, (p.value or 0), nb.value


def ka_three_phase_workspace_size(capacity: int):
    out = ctypes.c_uint64(0)
    s = lib.ka_three_phase_workspace_size(capacity, ctypes.byref(out))
    return s, out.value


def ka_compact_three_phase(d_in, n: int, d_n, pred: int, param: int, xform: int, d_out, d_count, d_ws,
                           ws_bytes: int, stream=None) -> int:
    return lib.ka_compact_three_phase(ptr(d_in), n, ptr(d_n), pred, param, xform, ptr(d_out), ptr(d_count),
                                      ptr(d_ws), ws_bytes, stream_ptr(stream))


KA_HOST_MAX_PRED = 4


def ka_compact_host_scratch_size(chunk: int, n_pred: int):
    out = ctypes.c_uint64(0)
    s = lib.ka_compact_host_scratch_size(chunk, n_pred, ctypes.byref(out))
    return s, out.value


def ka_compact_host(h_in, n: int, preds, params, xforms, h_outs, chunk: int, d_scratch, scratch_bytes: int):
    """Streamed compaction of host memory for len(preds) predicates; returns
    (status, [count per predicate])."""
    k = len(preds)
    pa = (ctypes.c_int32 * k)(*preds)
    qa = (ctypes.c_uint32 * k)(*params)
    xa = (ctypes.c_uint32 * k)(*xforms)
    oa = (c_vp * k)(*[ptr(o) for o in h_outs])
    ca = (ctypes.c_uint64 * k)()
    s = lib.ka_compact_host(ptr(h_in), n, k, pa, qa, xa, oa, ca, chunk, ptr(d_scratch), scratch_bytes)
    return s, [int(c) for c in ca]


def ka_mandelbrot(d_out, width: int, height: int, re_min: float, im_min: float, re_max: float, im_max: float,
                  max_iter: int, stream=None) -> int:
    return lib.ka_mandelbrot(ptr(d_out), width, height, re_min, im_min, re_max, im_max, max_iter,
                             stream_ptr(stream))


def ka_prepare_index(d_chunk_ids, d_literals, k: int, d_k, d_index, d_n_out=None, stream=None) -> int:
    return lib.ka_prepare_index(ptr(d_chunk_ids), ptr(d_literals), k, ptr(d_k), ptr(d_index), ptr(d_n_out),
                                stream_ptr(stream))


def ka_batch_workspace_size(max_items: int, total_capacity: int, tile=None):
    out = ctypes.c_uint64(0)
    s = lib.ka_batch_workspace_size(max_items, total_capacity, _tile(tile), ctypes.byref(out))
    return s, out.value


def ka_compact_batch(d_items, n_items: int, max_items: int, d_ws, ws_bytes: int, tile=None, grid: int = 0,
                     stream=None) -> int:
    return lib.ka_compact_batch(ptr(d_items), n_items, max_items, ptr(d_ws), ws_bytes, _tile(tile), grid,
                                stream_ptr(stream))


def ka_generate_batch(d_items, n_items: int, max_items: int, d_ws, ws_bytes: int, stream=None) -> int:
    return lib.ka_generate_batch(ptr(d_items), n_items, max_items, ptr(d_ws), ws_bytes, stream_ptr(stream))


def ka_autotune(kernel: int, n: int, cache_path=None, stream=None):
    best = ka_tile(0, 0)
    us = ctypes.c_float(0)
    s = lib.ka_autotune(kernel, n, cache_path.encode() if cache_path else None, ctypes.byref(best),
                        ctypes.byref(us), stream_ptr(stream))
    return s, (best.block, best.ipt), us.value


def ka_tile_for(kernel: int, n: int):
    t = ka_tile(0, 0)
    s = lib.ka_tile_for(kernel, n, ctypes.byref(t))
    return s, (t.block, t.ipt)


def ka_debug_device_cache(devices, values):
    """(status, [value each lookup returned]) for the per-device cache hook."""
    n = len(devices)
    d = (ctypes.c_int32 * n)(*devices)
    v = (ctypes.c_int32 * n)(*values)
    o = (ctypes.c_int32 * n)()
    s = lib.ka_debug_device_cache(d, v, n, o)
    return s, list(o)


def ka_debug_pred_keep(pred: int, param: int, x: int):
    out = ctypes.c_int32(0)
    s = lib.ka_debug_pred_keep(pred, param, x, ctypes.byref(out))
    return s, out.value


def ka_autotune_load(cache_path: str) -> int:
    return lib.ka_autotune_load(cache_path.encode())


# ---------------------------------------------------------------------------
# Actor layer (handles are opaque ints).
# ---------------------------------------------------------------------------
def ka_system_create(device: int = 0, stream=None, budget_bytes: int = 0, autotune_cache=None, debug: int = 0):
    cfg = ka_config(device, debug, stream_ptr(stream), budget_bytes,
                    autotune_cache.encode() if autotune_cache else None)
    h = c_vp(None)
    s = lib.ka_system_create(ctypes.byref(cfg), ctypes.byref(h))
    return s, h.value


def ka_system_destroy(sys_h, force: int = 0) -> int:
    return lib.ka_system_destroy(sys_h, force)


def ka_system_pool_bytes(sys_h):
    a, b = ctypes.c_uint64(0), ctypes.c_uint64(0)
    s = lib.ka_system_pool_bytes(sys_h, ctypes.byref(a), ctypes.byref(b))
    return s, a.value, b.value


def ka_ref_wrap(sys_h, d_ptr, n: int, capacity: int, dtype: int = KA_U32, access: int = KA_READ_WRITE):
    h = c_vp(None)
    s = lib.ka_ref_wrap(sys_h, ptr(d_ptr), n, capacity, dtype, access, ctypes.byref(h))
    return s, h.value


def ka_ref_alloc(sys_h, capacity: int, dtype: int = KA_U32):
    h = c_vp(None)
    s = lib.ka_ref_alloc(sys_h, capacity, dtype, ctypes.byref(h))
    return s, h.value


def ka_ref_count(ref_h):
    n = ctypes.c_uint64(0)
    s = lib.ka_ref_count(ref_h, ctypes.byref(n))
    return s, n.value


def ka_ref_info(ref_h):
    p, cap, dt, acc = c_vp(None), ctypes.c_uint64(0), ctypes.c_int32(0), ctypes.c_int32(0)
    s = lib.ka_ref_info(ref_h, ctypes.byref(p), ctypes.byref(cap), ctypes.byref(dt), ctypes.byref(acc))
    return s, p.value, cap.value, dt.value, acc.value


def ka_ref_retain(ref_h) -> int:
    return lib.ka_ref_retain(ref_h)


def ka_ref_release(ref_h) -> int:
    return lib.ka_ref_release(ref_h)


def ka_ref_serialize(ref_h, cap: int = 64):
    buf = ctypes.create_string_buffer(cap)
    n = ctypes.c_uint64(0)
    return lib.ka_ref_serialize(ref_h, buf, cap, ctypes.byref(n)), n.value


def ka_spawn_stage(sys_h, kind: int, pred: int = 0, param: int = 0, xform: int = 0, tile=(0, 0)):
    d = ka_stage_desc(kind, pred, param, xform, ka_tile(int(tile[0]), int(tile[1])))
    h = c_vp(None)
    s = lib.ka_spawn_stage(sys_h, ctypes.byref(d), ctypes.byref(h))
    return s, h.value


def ka_compose(b_h, a_h):
    h = c_vp(None)
    s = lib.ka_compose(b_h, a_h, ctypes.byref(h))
    return s, h.value


def ka_actor_arity(actor_h):
    i, o = ctypes.c_int32(0), ctypes.c_int32(0)
    s = lib.ka_actor_arity(actor_h, ctypes.byref(i), ctypes.byref(o))
    return s, i.value, o.value


def ka_actor_release(actor_h) -> int:
    return lib.ka_actor_release(actor_h)


def make_msg(refs=(), h_in=None, h_n: int = 0, h_out=None, h_out_cap: int = 0, seed: int = 0, gen_n: int = 0):
    """ka_msg for ka_request: device refs and/or host buffers (numpy uint32)."""
    m = ka_msg()
    m.n_refs = len(refs)
    for i, r in enumerate(refs):
        m.refs[i] = r
    if h_in is not None:
        m.h_in = h_in.ctypes.data_as(c_u32p)
        m.h_n = h_n if h_n else h_in.size
    if h_out is not None:
        m.h_out = h_out.ctypes.data_as(c_u32p)
        m.h_out_cap = h_out_cap if h_out_cap else h_out.size
    m.seed = seed & (2**64 - 1)
    m.gen_n = gen_n
    return m


def ka_request(actor_h, msg: ka_msg):
    h = c_vp(None)
    s = lib.ka_request(actor_h, ctypes.byref(msg), ctypes.byref(h))
    return s, h.value


def ka_receive(req_h, timeout_ns: int = -1):
    """Returns (status, msg): msg.refs[:msg.n_refs] are result ref handles."""
    m = ka_msg()
    s = lib.ka_receive(req_h, timeout_ns, ctypes.byref(m))
    return s, m


def ka_debug_fail_stage(actor_h, fail_after: int) -> int:
    return lib.ka_debug_fail_stage(actor_h, fail_after)


def ka_debug_kill_dispatcher(sys_h) -> int:
    return lib.ka_debug_kill_dispatcher(sys_h)


def ka_system_monitor(sys_h, fn, user=None) -> int:
    """fn(user, reason) is called once when the dispatcher dies; keep `fn` (a
    MONITOR_FN) alive while the system exists."""
    return lib.ka_system_monitor(sys_h, fn, user)


def ka_serve_run(sys_h, reqs, n_reqs: int, opt, results, stats) -> int:
    return lib.ka_serve_run(sys_h, reqs, n_reqs, ctypes.byref(opt), results, ctypes.byref(stats))


def serve_requests(arrival_s, n, seeds, stages):
    """Request array for ka_serve_run. stages[r] = [(pred, param, xform), ...]
    (1-4 entries) for request r."""
    arr = (ka_serve_request * len(n))()
    for r in range(len(n)):
        q = arr[r]
        q.arrival_s = float(arrival_s[r])
        q.seed = int(seeds[r]) & (2**64 - 1)
        q.n = int(n[r])
        q.n_stages = len(stages[r])
        for i, (pred, param, xform) in enumerate(stages[r]):
            q.stages[i] = ka_serve_stage(int(pred), int(param) & 0xFFFFFFFF, int(xform))
        q.h_out = None
        q.h_out_cap = 0
    return arr


KA_SERVE_BATCH_LONE = 1


def serve(sys_h, reqs, mode: int = 0, budget_bytes: int = 0, max_inflight: int = 0, time_scale: float = 1.0,
          tile=None, flags: int = 0):
    """Runs ka_serve_run; returns (status, results array, stats)."""
    opt = ka_serve_options(mode, max_inflight, budget_bytes, time_scale, ka_tile(*(tile or (0, 0))), flags)
    results = (ka_serve_result * max(len(reqs), 1))()
    stats = ka_serve_stats()
    st = lib.ka_serve_run(sys_h, reqs, len(reqs), ctypes.byref(opt), results, ctypes.byref(stats))
    return st, results, stats


def ka_bench_request_loop(actor_h, msg: ka_msg, iters: int, inflight: int = 1):
    sec, last = ctypes.c_double(0), ctypes.c_uint64(0)
    s = lib.ka_bench_request_loop(actor_h, ctypes.byref(msg), iters, inflight, ctypes.byref(sec), ctypes.byref(last))
    return s, sec.value, last.value


def stage_descs(specs):
    """[(kind, pred, param, xform), ...] -> ka_stage_desc array."""
    arr = (ka_stage_desc * len(specs))()
    for i, sp in enumerate(specs):
        kind, pred, param, xform = (tuple(sp) + (0, 0, 0))[:4]
        arr[i] = ka_stage_desc(kind, pred, param, xform, ka_tile(0, 0))
    return arr


KA_BENCH_WAIT_TAG = 1


def ka_bench_direct_chain(specs, d_in, n: int, iters: int, stream=None, flags: int = 0):
    arr = stage_descs(specs)
    sec, last = ctypes.c_double(0), ctypes.c_uint64(0)
    s = lib.ka_bench_direct_chain(arr, len(specs), ptr(d_in), n, iters, stream_ptr(stream), flags,
                                  ctypes.byref(sec), ctypes.byref(last))
    return s, sec.value, last.value
