"""A hand-built trace covering every case of device-activity pairing, with
its expected results written out by hand.

Host stream 0 (host "n0", pid 7, tid 7) makes launch / memcpy calls whose
ENTRY carries a 64-bit command id; device streams 1 and 2 (pid 900, tids 1
and 2) carry DEV_BEGIN / DEV_END events with command ids.  One case per
command:

  cmd        begins ends hosts  outcome
  A=0x0a      1     1    1      device interval, dur 50 (stream 1)
  B=0x0b      2     1    1      unpaired: two begins (3 device events)
  C=0x0c      1     1    1      unpaired: end before begin (2 events)
  D=0x0d      1     1    0      device pair, no host call: unjoined
  E=0x0e      1     1    2      device pair, two host calls: ambiguous
  F=0x0f      0     1    1      unpaired end (1 event)
  G=0x10      0     0    1      host call with no device work
  Z=0         1     1    1      device interval, dur 7 (stream 2; zero id)
  M=2^64-1    1     1    1      device interval, dur 30 (stream 2)
  (none)      1     0    0      DEV_BEGIN class without a command id: unpaired

Expected: dev_events 17, dev_pairs 5 (A, D, E, Z, M), dev_intervals 3
(A, Z, M), dev_unpaired 17 - 2*5 = 7 (B 3 + C 2 + F 1 + no-id 1),
dev_unjoined 1 (D), dev_ambiguous 1 (E), host_cmd_entries 9
(A, B, C, E twice, F, G, Z, M), host_unjoined 4 (B, C, F, G).
"""
from __future__ import annotations

import numpy as np

from tracegen.handbuilt import DEV_BEGIN, DEV_END, ENTRY, EXIT, Ev, TraceBuilder

A, B, C, D, E, F, G, Z, M = 0x0A, 0x0B, 0x0C, 0x0D, 0x0E, 0x0F, 0x10, 0, (1 << 64) - 1
T0 = 1_000_000


def build(packet_bytes: int = 256):
    tb = TraceBuilder(packet_bytes=packet_bytes)
    h = tb.add_host("n0")
    f_launch = tb.add_func("launchKernel")
    f_copy = tb.add_func("memcpyAsync")
    f_dev = tb.add_func("deviceWork", 3)
    # ENTRY classes carry the command id at offset 8 of a 16-byte fixed part
    e_launch = tb.add_class(f_launch, ENTRY, 16, cmd_off=8)
    x_launch = tb.add_class(f_launch, EXIT, 4, result_off=0)
    e_copy = tb.add_class(f_copy, ENTRY, 16, cmd_off=8)
    x_copy = tb.add_class(f_copy, EXIT, 4, result_off=0)
    c_begin = tb.add_class(f_dev, DEV_BEGIN, 8, cmd_off=0)
    c_end = tb.add_class(f_dev, DEV_END, 8, cmd_off=0)
    c_begin_noid = tb.add_class(f_dev, DEV_BEGIN, 8)
    s_host = tb.add_stream(h, 7, 7)
    s_d1 = tb.add_stream(h, 900, 1, 1)
    s_d2 = tb.add_stream(h, 900, 2, 1)

    def call(ent, ext, cmd, t, dur=10):
        return [Ev(ent, t, cmd=cmd), Ev(ext, t + dur, result=0)]

    host = []
    t = T0
    for cmd, (en, ex) in [(A, (e_launch, x_launch)), (B, (e_launch, x_launch)), (C, (e_copy, x_copy)),
                          (E, (e_launch, x_launch)), (E, (e_copy, x_copy)), (F, (e_launch, x_launch)),
                          (G, (e_copy, x_copy)), (Z, (e_launch, x_launch)), (M, (e_copy, x_copy))]:
        host += call(en, ex, cmd, t)
        t += 20
    d1 = [Ev(c_begin, T0 + 100, cmd=A), Ev(c_end, T0 + 150, cmd=A),
          Ev(c_begin, T0 + 160, cmd=B), Ev(c_end, T0 + 170, cmd=B), Ev(c_begin, T0 + 180, cmd=B),
          Ev(c_end, T0 + 185, cmd=C), Ev(c_begin, T0 + 190, cmd=C),
          Ev(c_begin, T0 + 200, cmd=D), Ev(c_end, T0 + 205, cmd=D),
          Ev(c_end, T0 + 210, cmd=F),
          Ev(c_begin_noid, T0 + 215)]
    d2 = [Ev(c_begin, T0 + 120, cmd=E), Ev(c_end, T0 + 125, cmd=E),
          Ev(c_begin, T0 + 130, cmd=Z), Ev(c_end, T0 + 137, cmd=Z),
          Ev(c_begin, T0 + 140, cmd=M), Ev(c_end, T0 + 170, cmd=M)]
    tb.place(tb.stream_events(s_host, host, ts_begin=T0))
    tb.place(tb.stream_events(s_d1, d1, ts_begin=T0))
    tb.place(tb.stream_events(s_d2, d2, ts_begin=T0))
    return tb.build(), dict(launch=f_launch, copy=f_copy, host=s_host, d1=s_d1, d2=s_d2)


EXPECTED_DEV_DIAG = dict(dev_events=17, dev_pairs=5, dev_intervals=3, dev_unpaired=7, dev_unjoined=1,
                         dev_ambiguous=1, host_cmd_entries=9, host_unjoined=4)


def expected_dev_rows(ids):
    """Device tally: A (launch, 50) on stream 1; Z (launch, 7) and M (memcpy, 30) on stream 2."""
    rows = [(0, 900, 1, ids["launch"], 1, 50, 50, 50, 0),
            (0, 900, 2, ids["launch"], 1, 7, 7, 7, 0),
            (0, 900, 2, ids["copy"], 1, 30, 30, 30, 0)]
    return sorted(rows)


def expected_dev_intervals(ids):
    """(start, end, stream, func, level, flags) of the three device intervals, by start."""
    return [(T0 + 100, T0 + 150, ids["d1"], ids["launch"], 0, 4),
            (T0 + 130, T0 + 137, ids["d2"], ids["launch"], 0, 4),
            (T0 + 140, T0 + 170, ids["d2"], ids["copy"], 0, 4)]


def as_tuples(arr: np.ndarray):
    return [tuple(int(v) for v in r) for r in arr.tolist()]
