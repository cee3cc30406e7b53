"""Thin ctypes binding of libthapi.so (argument marshalling only).

Every function mirrors the C ABI of include/thapi.h under the same name and
raises ThapiError on a non-zero status.  All analysis runs in the CUDA
library; if the library is missing, loading it raises (there is no CPU
fallback).  PyTorch is used only to supply device memory (the caching
allocator, through the context's allocator hooks) and streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libthapi.so")

OK, E_INVALID, E_FORMAT, E_TRUNCATED, E_NOMEM, E_TIMEOUT, E_CUDA, E_RANGE, E_UNSUPPORTED, PENDING = range(10)
REQ_LOAD, REQ_TALLY, REQ_WINDOW, REQ_FREE = range(4)  # serving-loop request kinds

ROW_DTYPE = np.dtype([("host_id", "<u4"), ("pid", "<u4"), ("tid", "<u4"), ("func_id", "<u4"),
                      ("count", "<u8"), ("total_ns", "<u8"), ("min_ns", "<u8"), ("max_ns", "<u8"),
                      ("err_count", "<u8")])
INTERVAL_DTYPE = np.dtype([("start_ns", "<u8"), ("end_ns", "<u8"), ("stream_id", "<u4"),
                           ("func_id", "<u2"), ("level", "u1"), ("flags", "u1")])
EVENT_DTYPE = np.dtype([("ts", "<u8"), ("cmd", "<u8"), ("stream_id", "<u4"), ("class_id", "<u2"),
                        ("var_len", "<u2"), ("result", "<i4"), ("ext", "u1"), ("kind", "u1"), ("func_id", "<u2"),
                        ("vpid", "<u4"), ("vtid", "<u4")])
DIAG_FIELDS = ("events", "pairs", "unmatched_entries", "unmatched_exits", "mismatched_pairs",
               "other_events", "discarded", "packets")
DEVICE_DIAG_FIELDS = ("dev_events", "dev_pairs", "dev_intervals", "dev_unpaired", "dev_unjoined", "dev_ambiguous",
                      "host_cmd_entries", "host_unjoined")
IV_ERR, IV_DEVICE = 1, 4  # interval flags

EXPORTED = (
    "thapi_ctx_create", "thapi_ctx_set_allocator", "thapi_ctx_destroy", "thapi_trace_load",
    "thapi_trace_load_device", "thapi_trace_free", "thapi_tally", "thapi_timeline", "thapi_tally_device",
    "thapi_timeline_device", "thapi_trace_info_get", "thapi_trace_strings", "thapi_last_error_location",
    "thapi_strerror", "thapi_ctx_set_timing", "thapi_trace_timing", "thapi_kernel_launches",
    "thapi_tally_static", "thapi_device_tally", "thapi_tally_merge", "thapi_decode", "thapi_ctx_set_self_time",
    "thapi_self_tally", "thapi_trace_func_layer", "thapi_trace_load_batch", "thapi_check_device_wait",
    "thapi_ctx_set_autotune", "thapi_server_create", "thapi_server_submit", "thapi_server_poll",
    "thapi_server_release", "thapi_server_now", "thapi_server_replay", "thapi_server_stats_get",
    "thapi_server_destroy",
)


class Diag(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in DIAG_FIELDS]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f in DIAG_FIELDS}


class DeviceDiag(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in DEVICE_DIAG_FIELDS]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f in DEVICE_DIAG_FIELDS}


class TraceInfo(ctypes.Structure):
    _fields_ = [("nbytes", ctypes.c_uint64), ("n_packets", ctypes.c_uint64), ("events", ctypes.c_uint64),
                ("intervals", ctypes.c_uint64), ("tally_rows", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                ("n_streams", ctypes.c_uint32), ("n_classes", ctypes.c_uint32), ("n_funcs", ctypes.c_uint32),
                ("n_hosts", ctypes.c_uint32), ("packet_bytes", ctypes.c_uint32), ("self_time", ctypes.c_uint32),
                ("t_min", ctypes.c_uint64), ("t_max", ctypes.c_uint64),
                ("device_rows", ctypes.c_uint64), ("device_intervals", ctypes.c_uint64)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class LoadTiming(ctypes.Structure):
    _fields_ = [(f, ctypes.c_float) for f in ("index_ms", "analyze_ms", "frontier_ms", "tally_ms", "compact_ms",
                                               "sort_ms", "gather_ms", "total_ms")] + \
               [(f, ctypes.c_uint64) for f in ("analyze_read_bytes", "analyze_write_bytes", "analyze_launches",
                                                "launches")] + \
               [(f, ctypes.c_float) for f in ("join_ms", "self_ms", "percpu_ms", "percpu_decode_ms")] + \
               [(f, ctypes.c_uint64) for f in ("percpu_read_bytes", "percpu_write_bytes")] + \
               [("grid_mult", ctypes.c_uint32), ("part_shift", ctypes.c_int32)] + \
               [(f, ctypes.c_float) for f in ("parse_ms", "call_ms")]

    def as_dict(self):
        return {f: (float(getattr(self, f)) if t is ctypes.c_float else int(getattr(self, f)))
                for f, t in self._fields_}


class Request(ctypes.Structure):
    """thapi_request (72 B)."""
    _fields_ = [("kind", ctypes.c_uint32), ("on_device", ctypes.c_uint32), ("bytes", ctypes.c_void_p),
                ("nbytes", ctypes.c_uint64), ("trace", ctypes.c_uint64), ("after", ctypes.c_uint64),
                ("t0", ctypes.c_uint64), ("t1", ctypes.c_uint64), ("out", ctypes.c_void_p), ("cap", ctypes.c_uint64)]


class Result(ctypes.Structure):
    """thapi_result (72 B)."""
    _fields_ = [("status", ctypes.c_int32), ("kind", ctypes.c_uint32), ("trace", ctypes.c_uint64),
                ("n", ctypes.c_uint64), ("events", ctypes.c_uint64), ("data", ctypes.c_void_p),
                ("t_arrival", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in ("submitted", "completed", "load_waits", "peak_running",
                                                "peak_committed", "result_allocs")]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p)

_lib = None


class ThapiError(RuntimeError):
    def __init__(self, code: int, where: str, location=None):
        self.code = code
        self.location = location
        super().__init__("%s: %s (status %d)%s" % (where, strerror(code) if _lib else "?", code,
                                                   "" if location is None else " at %r" % (location,)))


def library():
    """Loads libthapi.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libthapi.so is not built (run paper_2504_03683_b300.build.build())")
    lib = ctypes.CDLL(LIB_PATH)
    vp, u64, i32, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32
    P = ctypes.POINTER
    sig = {
        "thapi_ctx_create": ([P(vp), i32, u64], i32),
        "thapi_ctx_set_allocator": ([vp, ALLOC_FN, FREE_FN, vp], i32),
        "thapi_ctx_destroy": ([vp], i32),
        "thapi_trace_load": ([vp, vp, u64, vp, P(u64)], i32),
        "thapi_trace_load_device": ([vp, vp, u64, vp, P(u64)], i32),
        "thapi_trace_free": ([vp, u64], i32),
        "thapi_tally": ([vp, u64, vp, u64, P(u64), P(Diag)], i32),
        "thapi_tally_device": ([vp, u64, vp, u64, P(u64), P(Diag), vp], i32),
        "thapi_timeline": ([vp, u64, u64, u64, vp, u64, P(u64)], i32),
        "thapi_timeline_device": ([vp, u64, u64, u64, vp, u64, P(u64), vp], i32),
        "thapi_trace_info_get": ([vp, u64, P(TraceInfo)], i32),
        "thapi_trace_strings": ([vp, u64, i32, u32, ctypes.c_char_p, u64, P(u64)], i32),
        "thapi_last_error_location": ([vp, P(i32), P(u64), P(u64)], i32),
        "thapi_strerror": ([i32], ctypes.c_char_p),
        "thapi_ctx_set_timing": ([vp, i32], i32),
        "thapi_ctx_set_self_time": ([vp, i32], i32),
        "thapi_self_tally": ([vp, u64, vp, u64, P(u64)], i32),
        "thapi_trace_func_layer": ([vp, u64, u32, P(u32)], i32),
        "thapi_trace_load_batch": ([vp, vp, vp, u32, i32, vp, P(u64)], i32),
        "thapi_check_device_wait": ([vp, u32, vp], i32),
        "thapi_ctx_set_autotune": ([vp, i32], i32),
        "thapi_trace_timing": ([vp, u64, P(LoadTiming)], i32),
        "thapi_kernel_launches": ([], u64),
        "thapi_tally_static": ([vp, u64, vp, u64, P(u64), P(Diag), vp], i32),
        "thapi_device_tally": ([vp, u64, vp, u64, P(u64), P(DeviceDiag)], i32),
        "thapi_tally_merge": ([vp, vp, u64, vp, u64, P(u64), vp], i32),
        "thapi_decode": ([vp, vp, u64, vp, u64, P(u64), vp], i32),
        "thapi_server_create": ([vp, u32, u32, u64, P(vp)], i32),
        "thapi_server_submit": ([vp, P(Request), P(u64)], i32),
        "thapi_server_poll": ([vp, u64, u32, P(Result)], i32),
        "thapi_server_release": ([vp, u64], i32),
        "thapi_server_now": ([vp], ctypes.c_double),
        "thapi_server_replay": ([vp, P(Request), P(ctypes.c_double), u64, i32, P(Result)], i32),
        "thapi_server_stats_get": ([vp, P(ServerStats)], i32),
        "thapi_server_destroy": ([vp], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return library().thapi_strerror(code).decode()


def _check(code: int, where: str, ctx=None):
    if code != OK:
        loc = None
        if ctx is not None and code in (E_FORMAT, E_TRUNCATED):
            loc = thapi_last_error_location(ctx)
        raise ThapiError(code, where, loc)


def _stream_ptr(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# --------------------------------------------------------- C ABI mirrors
def thapi_ctx_create(device: int = 0, hbm_cap_bytes: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(library().thapi_ctx_create(ctypes.byref(h), device, hbm_cap_bytes), "thapi_ctx_create")
    return h.value


def thapi_ctx_set_allocator(ctx: int, alloc_fn, free_fn, user=None) -> None:
    _check(library().thapi_ctx_set_allocator(ctx, alloc_fn, free_fn, user), "thapi_ctx_set_allocator")


def thapi_ctx_destroy(ctx: int) -> None:
    _check(library().thapi_ctx_destroy(ctx), "thapi_ctx_destroy")


def thapi_trace_load(ctx: int, trace, stream=None) -> int:
    """Loads a trace from host memory (bytes, numpy uint8 array, or (address, nbytes))."""
    if isinstance(trace, tuple):
        ptr, n = trace
        keep = None
    elif isinstance(trace, np.ndarray):
        keep = np.ascontiguousarray(trace)
        ptr, n = keep.ctypes.data, keep.nbytes
    else:
        keep = np.frombuffer(trace, dtype=np.uint8)
        ptr, n = keep.ctypes.data, keep.nbytes
    tid = ctypes.c_uint64()
    rc = library().thapi_trace_load(ctx, ctypes.c_void_p(ptr), n, ctypes.c_void_p(_stream_ptr(stream)),
                                    ctypes.byref(tid))
    del keep
    _check(rc, "thapi_trace_load", ctx)
    return tid.value


def thapi_trace_load_device(ctx: int, dev_ptr: int, nbytes: int, stream=None) -> int:
    tid = ctypes.c_uint64()
    rc = library().thapi_trace_load_device(ctx, ctypes.c_void_p(dev_ptr), nbytes,
                                           ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(tid))
    _check(rc, "thapi_trace_load_device", ctx)
    return tid.value


def thapi_decode(ctx: int, trace, stream=None) -> np.ndarray:
    """Every event of a trace in host memory as an EVENT_DTYPE array (stream order)."""
    lib = library()
    arr = trace if isinstance(trace, np.ndarray) else np.frombuffer(trace, dtype=np.uint8)
    arr = np.ascontiguousarray(arr)
    n = ctypes.c_uint64()
    sp = ctypes.c_void_p(_stream_ptr(stream))
    code = lib.thapi_decode(ctx, arr.ctypes.data, arr.nbytes, None, 0, ctypes.byref(n), sp)
    if code != 0:
        _check(code, "thapi_decode", ctx)
    out = np.zeros(n.value, dtype=EVENT_DTYPE)
    if n.value:
        _check(lib.thapi_decode(ctx, arr.ctypes.data, arr.nbytes, out.ctypes.data, n.value, ctypes.byref(n), sp),
               "thapi_decode", ctx)
    return out


def thapi_trace_free(ctx: int, trace_id: int) -> None:
    _check(library().thapi_trace_free(ctx, trace_id), "thapi_trace_free")


def thapi_tally(ctx: int, trace_id: int):
    """Returns (rows as ROW_DTYPE array, diag dict)."""
    lib = library()
    n = ctypes.c_uint64()
    d = Diag()
    _check(lib.thapi_tally(ctx, trace_id, None, 0, ctypes.byref(n), ctypes.byref(d)), "thapi_tally")
    rows = np.zeros(n.value, dtype=ROW_DTYPE)
    if n.value:
        _check(lib.thapi_tally(ctx, trace_id, rows.ctypes.data, n.value, ctypes.byref(n), ctypes.byref(d)),
               "thapi_tally")
    return rows, d.as_dict()


def thapi_device_tally(ctx: int, trace_id: int):
    """Returns (device tally rows as ROW_DTYPE array, device diag dict)."""
    lib = library()
    n = ctypes.c_uint64()
    d = DeviceDiag()
    _check(lib.thapi_device_tally(ctx, trace_id, None, 0, ctypes.byref(n), ctypes.byref(d)), "thapi_device_tally")
    rows = np.zeros(n.value, dtype=ROW_DTYPE)
    if n.value:
        _check(lib.thapi_device_tally(ctx, trace_id, rows.ctypes.data, n.value, ctypes.byref(n), ctypes.byref(d)),
               "thapi_device_tally")
    return rows, d.as_dict()


def thapi_self_tally(ctx: int, trace_id: int):
    """Self-time rows (ROW_DTYPE: the tally's keys, counts and error counts;
    total / min / max of self time) of a trace loaded with self time on."""
    lib = library()
    n = ctypes.c_uint64()
    _check(lib.thapi_self_tally(ctx, trace_id, None, 0, ctypes.byref(n)), "thapi_self_tally")
    rows = np.zeros(n.value, dtype=ROW_DTYPE)
    if n.value:
        _check(lib.thapi_self_tally(ctx, trace_id, rows.ctypes.data, n.value, ctypes.byref(n)), "thapi_self_tally")
    return rows


def thapi_tally_merge(ctx: int, rows, stream=None):
    """Merges tally rows (ROW_DTYPE, any order; e.g. several traces' or ranks' rows
    concatenated) into one row per key, in key order."""
    lib = library()
    rows = np.ascontiguousarray(rows, dtype=ROW_DTYPE)
    n = ctypes.c_uint64()
    out = np.zeros(max(1, len(rows)), dtype=ROW_DTYPE)
    _check(lib.thapi_tally_merge(ctx, rows.ctypes.data if len(rows) else None, len(rows), out.ctypes.data, len(out),
                                 ctypes.byref(n), ctypes.c_void_p(_stream_ptr(stream))), "thapi_tally_merge")
    return out[: n.value].copy()


def thapi_tally_device(ctx: int, trace_id: int, dev_ptr: int, cap: int, stream=None):
    """Copies rows to device memory; returns (n_rows, diag dict)."""
    n = ctypes.c_uint64()
    d = Diag()
    _check(library().thapi_tally_device(ctx, trace_id, ctypes.c_void_p(dev_ptr), cap, ctypes.byref(n),
                                        ctypes.byref(d), ctypes.c_void_p(_stream_ptr(stream))),
           "thapi_tally_device")
    return n.value, d.as_dict()


def thapi_timeline(ctx: int, trace_id: int, t0: int = 0, t1: int = 2**64 - 1, out=None):
    """Returns the window's intervals as an INTERVAL_DTYPE array (into ``out`` if given)."""
    lib = library()
    n = ctypes.c_uint64()
    _check(lib.thapi_timeline(ctx, trace_id, t0, t1, None, 0, ctypes.byref(n)), "thapi_timeline")
    if out is None:
        out = np.zeros(n.value, dtype=INTERVAL_DTYPE)
    else:
        assert out.dtype == INTERVAL_DTYPE and out.flags["C_CONTIGUOUS"]
    if n.value:
        _check(lib.thapi_timeline(ctx, trace_id, t0, t1, out.ctypes.data, len(out), ctypes.byref(n)),
               "thapi_timeline")
    return out[: n.value]


def thapi_timeline_device(ctx: int, trace_id: int, t0: int, t1: int, dev_ptr: int, cap: int, stream=None) -> int:
    n = ctypes.c_uint64()
    _check(library().thapi_timeline_device(ctx, trace_id, t0, t1, ctypes.c_void_p(dev_ptr), cap, ctypes.byref(n),
                                           ctypes.c_void_p(_stream_ptr(stream))), "thapi_timeline_device")
    return n.value


def thapi_trace_info_get(ctx: int, trace_id: int) -> dict:
    info = TraceInfo()
    _check(library().thapi_trace_info_get(ctx, trace_id, ctypes.byref(info)), "thapi_trace_info_get")
    return info.as_dict()


def thapi_trace_strings(ctx: int, trace_id: int, kind: int, index: int) -> str:
    n = ctypes.c_uint64()
    rc = library().thapi_trace_strings(ctx, trace_id, kind, index, None, 0, ctypes.byref(n))
    if rc not in (OK, E_RANGE):
        _check(rc, "thapi_trace_strings")
    buf = ctypes.create_string_buffer(n.value + 1)
    _check(library().thapi_trace_strings(ctx, trace_id, kind, index, buf, n.value + 1, ctypes.byref(n)),
           "thapi_trace_strings")
    return buf.value.decode()


def thapi_last_error_location(ctx: int):
    lvl, pk, ev = ctypes.c_int(), ctypes.c_uint64(), ctypes.c_uint64()
    library().thapi_last_error_location(ctx, ctypes.byref(lvl), ctypes.byref(pk), ctypes.byref(ev))
    return (lvl.value, pk.value, ev.value)


def thapi_strerror(code: int) -> str:
    return strerror(code)


def thapi_ctx_set_timing(ctx: int, enable: bool = True) -> None:
    _check(library().thapi_ctx_set_timing(ctx, 1 if enable else 0), "thapi_ctx_set_timing")


def thapi_trace_load_batch(ctx: int, traces, stream=None, on_device: bool = False) -> int:
    """Loads several traces as one (see include/thapi.h).  traces: host buffers
    (bytes / uint8 arrays), or with on_device (device pointer, nbytes) pairs."""
    n = len(traces)
    ptrs = (ctypes.c_void_p * max(n, 1))()
    sizes = (ctypes.c_uint64 * max(n, 1))()
    keep = []
    for i, t in enumerate(traces):
        if on_device:
            ptrs[i], sizes[i] = int(t[0]), int(t[1])
        else:
            a = np.frombuffer(t, dtype=np.uint8) if isinstance(t, (bytes, bytearray)) else np.ascontiguousarray(t, dtype=np.uint8)
            keep.append(a)
            ptrs[i], sizes[i] = a.ctypes.data, a.nbytes
    out = ctypes.c_uint64()
    rc = library().thapi_trace_load_batch(ctx, ptrs, sizes, n, 1 if on_device else 0,
                                          ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(out))
    del keep
    _check(rc, "thapi_trace_load_batch", ctx)
    return int(out.value)


def thapi_check_device_wait(ctx: int, limit: int = 1024, stream=None) -> int:
    """Status code of a bounded device wait made to run out (THAPI_E_TIMEOUT expected)."""
    return int(library().thapi_check_device_wait(ctx, limit, ctypes.c_void_p(_stream_ptr(stream))))


def thapi_trace_func_layer(ctx: int, trace_id: int, func_id: int) -> int:
    v = ctypes.c_uint32()
    _check(library().thapi_trace_func_layer(ctx, trace_id, func_id, ctypes.byref(v)), "thapi_trace_func_layer")
    return int(v.value)


def thapi_ctx_set_autotune(ctx: int, enable: bool = True) -> None:
    _check(library().thapi_ctx_set_autotune(ctx, 1 if enable else 0), "thapi_ctx_set_autotune")


def thapi_ctx_set_self_time(ctx: int, enable: bool = True) -> None:
    _check(library().thapi_ctx_set_self_time(ctx, 1 if enable else 0), "thapi_ctx_set_self_time")


def thapi_trace_timing(ctx: int, trace_id: int) -> dict:
    t = LoadTiming()
    _check(library().thapi_trace_timing(ctx, trace_id, ctypes.byref(t)), "thapi_trace_timing")
    return t.as_dict()


def thapi_kernel_launches() -> int:
    return int(library().thapi_kernel_launches())


def thapi_tally_static(dev_ptr: int, nbytes: int, rows_dev_ptr: int, cap: int, stream=None):
    """Tally of a device-resident trace using only the library's static device
    scratch (for callers that must not allocate device memory); rows go to
    device memory.  Returns (n_rows, diag dict)."""
    n = ctypes.c_uint64()
    d = Diag()
    _check(library().thapi_tally_static(ctypes.c_void_p(dev_ptr), nbytes, ctypes.c_void_p(rows_dev_ptr), cap,
                                        ctypes.byref(n), ctypes.byref(d), ctypes.c_void_p(_stream_ptr(stream))),
           "thapi_tally_static")
    return n.value, d.as_dict()


# ------------------------------------------------- serving loop
def thapi_server_create(ctx: int, load_slots: int = 2, query_slots: int = 4, result_bytes: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(library().thapi_server_create(ctx, load_slots, query_slots, result_bytes, ctypes.byref(h)),
           "thapi_server_create")
    return h.value


def thapi_server_submit(srv: int, req: Request) -> int:
    t = ctypes.c_uint64()
    _check(library().thapi_server_submit(srv, ctypes.byref(req), ctypes.byref(t)), "thapi_server_submit")
    return int(t.value)


def thapi_server_poll(srv: int, ticket: int, wait_ms: int = 0xFFFFFFFF):
    """The request's Result, or None if it has not completed within wait_ms."""
    r = Result()
    rc = library().thapi_server_poll(srv, ticket, wait_ms, ctypes.byref(r))
    if rc == PENDING:
        return None
    _check(rc, "thapi_server_poll")
    return r


def thapi_server_release(srv: int, ticket: int) -> None:
    _check(library().thapi_server_release(srv, ticket), "thapi_server_release")


def thapi_server_now(srv: int) -> float:
    return float(library().thapi_server_now(srv))


def thapi_server_replay(srv: int, reqs, arrivals, keep: bool = False):
    """Submits reqs[i] (Request) at arrivals[i] seconds from the call, waits for
    all; returns the list of Result."""
    n = len(reqs)
    arr_t = (Request * max(n, 1))(*reqs)
    at = (ctypes.c_double * max(n, 1))(*[float(a) for a in arrivals])
    res = (Result * max(n, 1))()
    _check(library().thapi_server_replay(srv, arr_t, at, n, 1 if keep else 0, res), "thapi_server_replay")
    return [res[i] for i in range(n)]


def thapi_server_stats_get(srv: int) -> dict:
    st = ServerStats()
    _check(library().thapi_server_stats_get(srv, ctypes.byref(st)), "thapi_server_stats_get")
    return st.as_dict()


def thapi_server_destroy(srv: int) -> None:
    _check(library().thapi_server_destroy(srv), "thapi_server_destroy")


def result_rows(res: Result) -> np.ndarray:
    """A TALLY result's rows (a copy of the result memory)."""
    if res.status != OK or not res.n:
        return np.zeros(0, dtype=ROW_DTYPE)
    return np.ctypeslib.as_array(ctypes.cast(res.data, ctypes.POINTER(ctypes.c_uint8)),
                                 (res.n * ROW_DTYPE.itemsize,)).view(ROW_DTYPE).copy()


def result_intervals(res: Result) -> np.ndarray:
    """A WINDOW result's intervals (a copy of the result memory)."""
    if res.status != OK or not res.n:
        return np.zeros(0, dtype=INTERVAL_DTYPE)
    return np.ctypeslib.as_array(ctypes.cast(res.data, ctypes.POINTER(ctypes.c_uint8)),
                                 (res.n * INTERVAL_DTYPE.itemsize,)).view(INTERVAL_DTYPE).copy()


# ------------------------------------------------- torch device memory
class TorchAllocator:
    """Allocator hooks that route the library's device memory to torch's caching allocator."""

    def __init__(self, device: int = 0):
        import torch  # plumbing only

        self._torch = torch
        self.device = device

        def _alloc(nbytes, stream, _user):
            try:
                return self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device, int(stream or 0))
            except Exception:
                return None

        def _free(ptr, _nbytes, _stream, _user):
            try:
                self._torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:
                pass

        self.alloc_fn = ALLOC_FN(_alloc)
        self.free_fn = FREE_FN(_free)


class Context:
    """Owns a thapi context on one device, with torch-backed device memory."""

    def __init__(self, device: int = 0, hbm_cap_bytes: int = 0, use_torch_allocator: bool = True):
        self.device = device
        self.handle = thapi_ctx_create(device, hbm_cap_bytes)
        self._alloc = None
        if use_torch_allocator:
            self._alloc = TorchAllocator(device)
            thapi_ctx_set_allocator(self.handle, self._alloc.alloc_fn, self._alloc.free_fn)

    def load(self, trace, stream=None) -> int:
        return thapi_trace_load(self.handle, trace, stream)

    def load_batch(self, traces, stream=None) -> int:
        return thapi_trace_load_batch(self.handle, traces, stream)

    def load_batch_device(self, ptr_sizes, stream=None) -> int:
        return thapi_trace_load_batch(self.handle, ptr_sizes, stream, on_device=True)

    def load_device(self, dev_ptr: int, nbytes: int, stream=None) -> int:
        return thapi_trace_load_device(self.handle, dev_ptr, nbytes, stream)

    def tally(self, trace_id: int):
        return thapi_tally(self.handle, trace_id)

    def decode(self, trace, stream=None):
        return thapi_decode(self.handle, trace, stream)

    def device_tally(self, trace_id: int):
        return thapi_device_tally(self.handle, trace_id)

    def tally_merge(self, rows, stream=None):
        return thapi_tally_merge(self.handle, rows, stream)

    def set_self_time(self, enable: bool = True) -> None:
        thapi_ctx_set_self_time(self.handle, enable)

    def self_tally(self, trace_id: int):
        return thapi_self_tally(self.handle, trace_id)

    def timeline(self, trace_id: int, t0: int = 0, t1: int = 2**64 - 1):
        return thapi_timeline(self.handle, trace_id, t0, t1)

    def info(self, trace_id: int) -> dict:
        return thapi_trace_info_get(self.handle, trace_id)

    def free(self, trace_id: int) -> None:
        thapi_trace_free(self.handle, trace_id)

    def close(self) -> None:
        if self.handle:
            thapi_ctx_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
