"""Seeded synthetic THPT traces (input generator shared by tests and bench).

Holds none of the analysis arithmetic: it writes trace bytes and records what
it wrote (the per-call ground truth and the per-event list).  The CPU oracle
and the CUDA library both read what this module writes; neither imports the
other.

Presets follow the workloads the trace-analysis path is measured on: the
paper's analysis inputs are traces of intercepted API entry/exit events
(Sec. 3.2, Sec. 3.4) with layered APIs nesting on one thread (Sec. 4.3):

* ``tiny``    1 host, 1 pid, 4 threads; one API of 40 functions; 100k calls;
              depth <= 3; log-normal self time median 2 us; gaps 1 us;
              payloads 0-48 B; 4 KB packets.
* ``large``   8 hosts x 8 pids x 8 threads (512 streams); portable (60 fns)
              over vendor (120 fns) plus a message-passing layer (30 fns);
              100M calls (200M events, ~8 GB); depth <= 6; median 5 us;
              1 % error results; 16 KB packets.
* ``device``  8 hosts x 8 pids x 8 threads (512 host streams) of launch /
              memcpy calls (16 fns) carrying unique random 64-bit command
              ids; 64 device streams run each command after its submit
              (log-normal device time, median 400 ns, so the 8 host streams
              feeding one device stream keep it about half busy) and log
              DEV_BEGIN / DEV_END with the id; 50M commands = 200M events.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tracegen.cpp")
_LIB_PATH = os.path.join(_HERE, "libtracegen.so")
_lock = threading.Lock()
_lib = None

MODEL_FLAT = 1
MODEL_LAYERED = 2
MODEL_DEVICE = 4


class TgConfig(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("total_calls", ctypes.c_uint64),
        ("n_hosts", ctypes.c_uint32),
        ("pids_per_host", ctypes.c_uint32),
        ("tids_per_pid", ctypes.c_uint32),
        ("packet_bytes", ctypes.c_uint32),
        ("model", ctypes.c_uint32),
        ("max_depth", ctypes.c_uint32),
        ("n_flat", ctypes.c_uint32),
        ("n_portable", ctypes.c_uint32),
        ("n_vendor", ctypes.c_uint32),
        ("n_mpi", ctypes.c_uint32),
        ("var_min", ctypes.c_uint32),
        ("var_max", ctypes.c_uint32),
        ("n_threads", ctypes.c_uint32),
        ("n_device_streams", ctypes.c_uint32),
        ("dur_median_ns", ctypes.c_double),
        ("dur_sigma", ctypes.c_double),
        ("gap_mean_ns", ctypes.c_double),
        ("p_err", ctypes.c_double),
        ("p_drop", ctypes.c_double),
        ("p_long_gap", ctypes.c_double),
        ("long_gap_ns", ctypes.c_double),
        ("p_ext", ctypes.c_double),
        ("p_nest", ctypes.c_double),
        ("p_sample", ctypes.c_double),
        ("dev_dur_median_ns", ctypes.c_double),
        ("n_cpus", ctypes.c_uint32),       # > 0: per-CPU buffers (n_cpus per host), threads scheduled onto CPUs
        ("reserved", ctypes.c_uint32),
        ("slice_ns", ctypes.c_double),     # per-CPU scheduling time slice
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


CALL_DTYPE = np.dtype(
    [("start_ns", "<u8"), ("end_ns", "<u8"), ("stream_id", "<u4"), ("func_id", "<u2"),
     ("level", "u1"), ("flags", "u1")]
)
EVENT_DTYPE = np.dtype(
    [("ts", "<u8"), ("cmd", "<u8"), ("stream_id", "<u4"), ("class_id", "<u2"), ("var_len", "<u2"),
     ("result", "<i4"), ("ext", "u1"), ("kind", "u1"), ("func_id", "<u2")]
)
assert CALL_DTYPE.itemsize == 24 and EVENT_DTYPE.itemsize == 32

# ground-truth call flags
CALL_ERR = 1
CALL_ENTRY_DROPPED = 2
CALL_EXIT_DROPPED = 4
CALL_DEVICE = 8
CALL_HOST_DROPPED = 16  # device interval whose issuing host call lost its ENTRY event


def build(force: bool = False) -> str:
    """Compiles libtracegen.so next to its source (host code, g++)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    lib.tg_default_config.argtypes = [ctypes.POINTER(TgConfig)]
    lib.tg_default_config.restype = None
    lib.tg_plan_create.argtypes = [ctypes.POINTER(TgConfig)]
    lib.tg_plan_create.restype = ctypes.c_void_p
    lib.tg_plan_bytes.argtypes = [ctypes.c_void_p]
    lib.tg_plan_bytes.restype = ctypes.c_uint64
    lib.tg_plan_packets.argtypes = [ctypes.c_void_p]
    lib.tg_plan_packets.restype = ctypes.c_uint64
    lib.tg_plan_streams.argtypes = [ctypes.c_void_p]
    lib.tg_plan_streams.restype = ctypes.c_uint32
    lib.tg_plan_write.argtypes = [
        ctypes.c_void_p, ctypes.c_void_p,
        ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64),
        ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64),
    ]
    lib.tg_plan_write.restype = ctypes.c_int
    lib.tg_plan_destroy.argtypes = [ctypes.c_void_p]
    lib.tg_plan_destroy.restype = None
    _lib = lib
    return lib


def config(**overrides) -> TgConfig:
    """A TgConfig with library defaults, then ``overrides`` applied."""
    lib = _load()
    c = TgConfig()
    lib.tg_default_config(ctypes.byref(c))
    for k, v in overrides.items():
        if not hasattr(c, k):
            raise KeyError(k)
        setattr(c, k, v)
    return c


def preset(name: str, **overrides) -> TgConfig:
    """Named workload shapes; ``overrides`` (e.g. total_calls, seed) win."""
    if name == "tiny":
        base = dict(seed=0, total_calls=100_000, n_hosts=1, pids_per_host=1, tids_per_pid=4,
                    packet_bytes=4096, model=MODEL_FLAT, max_depth=3, n_flat=40,
                    dur_median_ns=2000.0, dur_sigma=1.0, gap_mean_ns=1000.0,
                    var_min=0, var_max=48, p_nest=0.3)
    elif name == "large":
        base = dict(seed=1, total_calls=100_000_000, n_hosts=8, pids_per_host=8, tids_per_pid=8,
                    packet_bytes=16384, model=MODEL_LAYERED, max_depth=6,
                    n_portable=60, n_vendor=120, n_mpi=30,
                    dur_median_ns=5000.0, dur_sigma=1.0, gap_mean_ns=1000.0,
                    var_min=0, var_max=48, p_err=0.01, p_nest=0.25)
    elif name == "device":
        base = dict(seed=2, total_calls=50_000_000, n_hosts=8, pids_per_host=8, tids_per_pid=8,
                    packet_bytes=16384, model=MODEL_DEVICE, max_depth=1, n_flat=16,
                    n_device_streams=64, dur_median_ns=5000.0, dur_sigma=1.0,
                    gap_mean_ns=1000.0, var_min=0, var_max=48, p_err=0.01, dev_dur_median_ns=400.0)
    elif name == "percpu":  # the large workload's calls written as per-CPU buffers (32 CPUs per host)
        base = dict(seed=1, total_calls=50_000_000, n_hosts=8, pids_per_host=8, tids_per_pid=8,
                    packet_bytes=16384, model=MODEL_LAYERED, max_depth=6,
                    n_portable=60, n_vendor=120, n_mpi=30,
                    dur_median_ns=5000.0, dur_sigma=1.0, gap_mean_ns=1000.0,
                    var_min=0, var_max=48, p_err=0.01, p_nest=0.25, n_cpus=32, slice_ns=200_000.0)
    else:
        raise KeyError(name)
    base.update(overrides)
    return config(**base)


class Plan:
    """Sizing pass done; ``write`` fills a caller buffer of ``nbytes``."""

    def __init__(self, cfg: TgConfig):
        self._lib = _load()
        self.cfg = cfg
        self._h = self._lib.tg_plan_create(ctypes.byref(cfg))
        if not self._h:
            raise ValueError("tracegen: invalid config %r" % (cfg.as_dict(),))
        self.nbytes = int(self._lib.tg_plan_bytes(self._h))
        self.n_packets = int(self._lib.tg_plan_packets(self._h))
        self.n_streams = int(self._lib.tg_plan_streams(self._h))

    def write(self, ptr: int, truth: bool = False):
        """Writes the trace at address ``ptr``; returns (calls, events) or (None, None)."""
        if not truth:
            rc = self._lib.tg_plan_write(self._h, ctypes.c_void_p(ptr), None, 0, None, None, 0, None)
            if rc != 0:
                raise RuntimeError("tracegen write failed")
            return None, None
        nc = ctypes.c_uint64(0)
        ne = ctypes.c_uint64(0)
        # first pass sizes the truth arrays (writes the bytes too; the second pass rewrites them identically)
        self._lib.tg_plan_write(self._h, ctypes.c_void_p(ptr), None, 0, ctypes.byref(nc), None, 0, ctypes.byref(ne))
        calls = np.zeros(nc.value, dtype=CALL_DTYPE)
        events = np.zeros(ne.value, dtype=EVENT_DTYPE)
        rc = self._lib.tg_plan_write(
            self._h, ctypes.c_void_p(ptr),
            calls.ctypes.data, nc.value, ctypes.byref(nc),
            events.ctypes.data, ne.value, ctypes.byref(ne))
        if rc != 0:
            raise RuntimeError("tracegen truth write failed")
        return calls, events

    def close(self):
        if self._h:
            self._lib.tg_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def generate(cfg: TgConfig, truth: bool = False):
    """Returns (bytes as np.uint8 array, calls, events); calls/events are None unless truth."""
    plan = Plan(cfg)
    buf = np.empty(plan.nbytes, dtype=np.uint8)
    calls, events = plan.write(buf.ctypes.data, truth=truth)
    plan.close()
    return buf, calls, events
