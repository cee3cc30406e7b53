"""THPT trace-analysis oracle (TEST INFRASTRUCTURE ONLY).

A plain sequential CPU statement of the analysis path (decode, per-thread
call-stack pairing, ordered-map tally, device-activity pairing by command id,
time-ordered timeline), compiled from ``oracle.cpp``.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the CUDA library never
does and shares no code with it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, E_INVALID, E_FORMAT, E_TRUNCATED = 0, 1, 2, 3

ROW_DTYPE = np.dtype([("host_id", "<u4"), ("pid", "<u4"), ("tid", "<u4"), ("func_id", "<u4"),
                      ("count", "<u8"), ("total_ns", "<u8"), ("min_ns", "<u8"), ("max_ns", "<u8"),
                      ("err_count", "<u8")])
INTERVAL_DTYPE = np.dtype([("start_ns", "<u8"), ("end_ns", "<u8"), ("stream_id", "<u4"),
                           ("func_id", "<u2"), ("level", "u1"), ("flags", "u1")])
EVENT_DTYPE = np.dtype([("ts", "<u8"), ("cmd", "<u8"), ("stream_id", "<u4"), ("class_id", "<u2"),
                        ("var_len", "<u2"), ("result", "<i4"), ("ext", "u1"), ("kind", "u1"),
                        ("func_id", "<u2"), ("vpid", "<u4"), ("vtid", "<u4")])
DIAG_FIELDS = ("events", "pairs", "unmatched_entries", "unmatched_exits", "mismatched_pairs",
               "other_events", "discarded", "packets")
DEV_DIAG_FIELDS = ("dev_events", "dev_pairs", "dev_intervals", "dev_unpaired", "dev_unjoined", "dev_ambiguous",
                   "host_cmd_entries", "host_unjoined")
IV_ERR, IV_DEVICE = 1, 4
assert ROW_DTYPE.itemsize == 56 and INTERVAL_DTYPE.itemsize == 24 and EVENT_DTYPE.itemsize == 40


class _Opts(ctypes.Structure):
    _fields_ = [("streams", ctypes.c_void_p), ("n_subset", ctypes.c_uint32),
                ("want_intervals", ctypes.c_uint32), ("t0", ctypes.c_uint64), ("t1", ctypes.c_uint64)]


class _Diag(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in DIAG_FIELDS]


class _DevDiag(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in DEV_DIAG_FIELDS]


def build(force: bool = False) -> str:
    """Compiles liboracle.so next to its source (host code, g++)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread", "-Wall", "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    vp, u64 = ctypes.c_void_p, ctypes.c_uint64
    lib.orc_run.argtypes = [vp, u64, ctypes.POINTER(_Opts), ctypes.POINTER(vp)]
    lib.orc_run.restype = ctypes.c_int
    lib.orc_run_threads.argtypes = [vp, u64, ctypes.POINTER(_Opts), ctypes.c_uint32, ctypes.POINTER(vp)]
    lib.orc_run_threads.restype = ctypes.c_int
    lib.orc_n_rows.argtypes = [vp]
    lib.orc_n_rows.restype = u64
    lib.orc_rows.argtypes = [vp]
    lib.orc_rows.restype = vp
    lib.orc_n_intervals.argtypes = [vp]
    lib.orc_n_intervals.restype = u64
    lib.orc_intervals.argtypes = [vp]
    lib.orc_intervals.restype = vp
    lib.orc_get_diag.argtypes = [vp, ctypes.POINTER(_Diag)]
    lib.orc_get_diag.restype = None
    lib.orc_n_dev_rows.argtypes = [vp]
    lib.orc_n_dev_rows.restype = u64
    lib.orc_dev_rows.argtypes = [vp]
    lib.orc_dev_rows.restype = vp
    lib.orc_n_self_rows.argtypes = [vp]
    lib.orc_n_self_rows.restype = u64
    lib.orc_self_rows.argtypes = [vp]
    lib.orc_self_rows.restype = vp
    lib.orc_get_dev_diag.argtypes = [vp, ctypes.POINTER(_DevDiag)]
    lib.orc_get_dev_diag.restype = None
    lib.orc_error_location.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(u64), ctypes.POINTER(u64)]
    lib.orc_error_location.restype = None
    lib.orc_free.argtypes = [vp]
    lib.orc_free.restype = None
    lib.orc_decode.argtypes = [vp, u64, vp, u64, ctypes.POINTER(u64)]
    lib.orc_decode.restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(buf):
    if isinstance(buf, np.ndarray):
        assert buf.flags["C_CONTIGUOUS"]
        return buf.ctypes.data, buf.nbytes, buf
    arr = np.frombuffer(buf, dtype=np.uint8)
    return arr.ctypes.data, arr.nbytes, arr


class Result:
    def __init__(self, code, loc, rows, intervals, diag, dev_rows, dev_diag, self_rows):
        self.code = code
        self.loc = loc            # (level, packet, event): 0 file, 1 packet header, 2 packet content
        self.rows = rows          # ROW_DTYPE, ordered by (host_id, pid, tid, func_id)
        self.intervals = intervals  # INTERVAL_DTYPE, timeline order (host and device intervals)
        self.diag = diag          # dict of DIAG_FIELDS
        self.dev_rows = dev_rows  # ROW_DTYPE: device intervals per (device stream's host, pid, tid; host function)
        self.dev_diag = dev_diag  # dict of DEV_DIAG_FIELDS
        self.self_rows = self_rows  # ROW_DTYPE, the rows' keys and counts; total / min / max of self time


def run(trace, streams=None, t0: int = 0, t1: int = 2**64 - 1, want_intervals: bool = True) -> Result:
    """Validates and analyses ``trace`` (bytes or uint8 array).

    ``streams`` restricts analysis (and validation) to those stream ids.
    """
    return _run(trace, streams, t0, t1, want_intervals, 1)


def _run(trace, streams, t0, t1, want_intervals, threads) -> Result:
    lib = _load()
    p, n, keep = _ptr(trace)
    opts = _Opts()
    sub = None
    if streams is not None:
        sub = np.ascontiguousarray(np.asarray(streams, dtype=np.uint32))
        opts.streams = sub.ctypes.data
        opts.n_subset = sub.size
    opts.want_intervals = 1 if want_intervals else 0
    opts.t0 = t0
    opts.t1 = t1
    h = ctypes.c_void_p()
    if threads > 1:
        code = lib.orc_run_threads(p, n, ctypes.byref(opts), threads, ctypes.byref(h))
    else:
        code = lib.orc_run(p, n, ctypes.byref(opts), ctypes.byref(h))
    try:
        lvl, pk, ev = ctypes.c_int(), ctypes.c_uint64(), ctypes.c_uint64()
        lib.orc_error_location(h, ctypes.byref(lvl), ctypes.byref(pk), ctypes.byref(ev))
        nr = lib.orc_n_rows(h)
        rows = np.zeros(nr, dtype=ROW_DTYPE)
        if nr:
            ctypes.memmove(rows.ctypes.data, lib.orc_rows(h), nr * ROW_DTYPE.itemsize)
        ni = lib.orc_n_intervals(h)
        ivs = np.zeros(ni, dtype=INTERVAL_DTYPE)
        if ni:
            ctypes.memmove(ivs.ctypes.data, lib.orc_intervals(h), ni * INTERVAL_DTYPE.itemsize)
        d = _Diag()
        lib.orc_get_diag(h, ctypes.byref(d))
        diag = {f: int(getattr(d, f)) for f in DIAG_FIELDS}
        nd = lib.orc_n_dev_rows(h)
        dev_rows = np.zeros(nd, dtype=ROW_DTYPE)
        if nd:
            ctypes.memmove(dev_rows.ctypes.data, lib.orc_dev_rows(h), nd * ROW_DTYPE.itemsize)
        ns = lib.orc_n_self_rows(h)
        self_rows = np.zeros(ns, dtype=ROW_DTYPE)
        if ns:
            ctypes.memmove(self_rows.ctypes.data, lib.orc_self_rows(h), ns * ROW_DTYPE.itemsize)
        dd = _DevDiag()
        lib.orc_get_dev_diag(h, ctypes.byref(dd))
        dev_diag = {f: int(getattr(dd, f)) for f in DEV_DIAG_FIELDS}
    finally:
        lib.orc_free(h)
    del keep, sub
    return Result(code, (lvl.value, pk.value, ev.value), rows, ivs, diag, dev_rows, dev_diag, self_rows)


def decode(trace) -> np.ndarray:
    """Every event in stream order (EVENT_DTYPE); raises on an invalid trace."""
    lib = _load()
    p, n, keep = _ptr(trace)
    cnt = ctypes.c_uint64()
    code = lib.orc_decode(p, n, None, 0, ctypes.byref(cnt))
    if code != OK:
        raise ValueError("invalid trace (code %d)" % code)
    out = np.zeros(cnt.value, dtype=EVENT_DTYPE)
    lib.orc_decode(p, n, out.ctypes.data, cnt.value, ctypes.byref(cnt))
    del keep
    return out



def run_threads(trace, threads: int, streams=None) -> Result:
    """The oracle on all host cores: ``orc_run_threads`` deals the streams round
    robin to `threads` std::threads, each running the plain definition on its
    subset, and merges the partial results (rows by key, diagnostics added,
    intervals merged by (start, stream)).  Exact for traces whose streams pair
    independently; traces with per-CPU buffers or device activity run on one
    thread.  For valid traces (an invalid subset reports its own location)."""
    return _run(trace, streams, 0, 2**64 - 1, True, threads)
