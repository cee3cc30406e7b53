"""A per-thread trace re-written as per-CPU buffers (input construction only).

Every thread of the input runs on the CPUs of its host: it starts on CPU
(tid mod n_cpus) and moves to another CPU after a random number of its events
(never between two of its events with the same timestamp, so that ordering a
thread's events by (ts, buffer, position) gives back its own order).  Each CPU
buffer is a stream of the output with flags bit 1 and holds the events of the
threads while they ran there, in time order, each event carrying its thread's
(vpid, vtid).  Pairing the threads of the output must give the tally of the
input and its intervals up to the stream they belong to.
"""
from __future__ import annotations

import random
import struct

import numpy as np

import oracle
from tracegen.handbuilt import Ev, TraceBuilder


def _tables(b: bytes):
    (magic, ver, hb, P, n_streams, n_classes, n_funcs, n_hosts, _z) = struct.unpack_from("<IHHIIIIII", b, 0)
    (n_packets, st_off, cl_off, fn_off, ho_off, str_off, str_bytes, pk_off) = struct.unpack_from("<8Q", b, 32)
    streams = [struct.unpack_from("<IIII", b, st_off + 16 * i) for i in range(n_streams)]
    classes = [struct.unpack_from("<HBBHhh", b, cl_off + 16 * i) for i in range(n_classes)]
    strings = b[str_off:str_off + str_bytes]

    def name(off):
        return strings[off:strings.index(b"\x00", off)].decode()
    funcs = [(name(struct.unpack_from("<I", b, fn_off + 8 * i)[0]), struct.unpack_from("<H", b, fn_off + 8 * i + 4)[0])
             for i in range(n_funcs)]
    hosts = [name(struct.unpack_from("<I", b, ho_off + 8 * i)[0]) for i in range(n_hosts)]
    return P, streams, classes, funcs, hosts


def to_per_cpu(trace, n_cpus: int = 4, seed: int = 0, mean_run: int = 40, packet_bytes: int | None = None):
    b = bytes(trace)
    P, streams, classes, funcs, hosts = _tables(b)
    ev = oracle.decode(trace)
    rng = random.Random(seed)
    tb = TraceBuilder(packet_bytes=packet_bytes or P)
    for h in hosts:
        tb.add_host(h)
    for (fname, layer) in funcs:
        tb.add_func(fname, layer)
    for (func, kind, _z, fixed, roff, coff) in classes:
        tb.add_class(func, kind, fixed, roff, coff)
    cpu_stream = {}
    for h in range(len(hosts)):
        for c in range(n_cpus):
            cpu_stream[(h, c)] = tb.add_stream(h, 0, c, 2)
    per_cpu = {k: [] for k in cpu_stream}
    for sid, (host, pid, tid, _f) in enumerate(streams):
        mine = ev[ev["stream_id"] == sid]
        cpu = tid % n_cpus
        left = rng.randint(1, 2 * mean_run)
        prev_ts = None
        for j in range(len(mine)):
            e = mine[j]
            ts = int(e["ts"])
            if left <= 0 and prev_ts is not None and ts > prev_ts:
                cpu = (cpu + rng.randint(1, n_cpus - 1)) % n_cpus if n_cpus > 1 else cpu
                left = rng.randint(1, 2 * mean_run)
            left -= 1
            prev_ts = ts
            per_cpu[(host, cpu)].append((ts, sid, j, Ev(int(e["class_id"]), ts, payload=b"\x00" * int(e["var_len"]),
                                                       result=int(e["result"]), cmd=int(e["cmd"]) or None,
                                                       ctx=(pid, tid))))
    for key, lst in per_cpu.items():
        lst.sort(key=lambda x: (x[0], x[1], x[2]))
        if lst:
            tb.place(tb.stream_events(cpu_stream[key], [x[3] for x in lst], ts_begin=lst[0][0]))
    return tb.build()
