"""Pins for the CPU oracle against facts fixed outside it.

* decode round trip against the generator's own record of what it wrote
  (timestamps, classes, results, command ids, EXT choice);
* tallies and timelines against the generator's ground-truth call list
  (a plain group-by / sort over calls the generator made, drop-free traces);
* brute force: every short entry/exit sequence, paired by the clamped-depth
  definition in O(n^2), versus the oracle's call stack;
* invariants on traces with dropped events;
* error codes and locations on malformed traces;
* the worked tally table of the paper (Sec. 4.3), reproduced at its printed
  precision (see test_paper_table.py).
"""
from __future__ import annotations

import itertools
import random
import struct

import numpy as np
import pytest

import oracle
import tracegen as tg
from tracegen.handbuilt import DEV_BEGIN, ENTRY, EXIT, SAMPLE, Ev, TraceBuilder
from tests._util import (brute_force_stream, expected_device_from_truth, expected_from_truth, intervals_equal,
                         merge_timelines, rows_equal,
                         stream_table, tally_from_pairs)


# ------------------------------------------------------------ round trip
@pytest.mark.parametrize("cfg", [
    dict(name="tiny"),
    dict(name="large", total_calls=30_000, p_long_gap=0.01, long_gap_ns=3e8, p_ext=0.01, p_sample=0.05,
         packet_bytes=1024),
    dict(name="device", total_calls=20_000, n_hosts=1, pids_per_host=2, tids_per_pid=2, n_device_streams=3),
])
def test_decode_roundtrip(cfg):
    cfg = dict(cfg)
    name = cfg.pop("name")
    b, _calls, ev = tg.generate(tg.preset(name, **cfg), truth=True)
    d = oracle.decode(b)
    assert len(d) == len(ev)
    for f in ("ts", "cmd", "stream_id", "class_id", "var_len", "result", "ext", "kind", "func_id"):
        assert np.array_equal(d[f], ev[f]), f
    if name == "large":
        assert ev["ext"].sum() > 0


def test_ext_boundary_deltas():
    tb = TraceBuilder(packet_bytes=256)
    h = tb.add_host("h")
    f, e, x = tb.add_call_func("f")
    s = tb.add_stream(h, 1, 1)
    t0 = 10**18
    evs = [Ev(e, t0), Ev(x, t0 + (1 << 27) - 1), Ev(e, t0 + (1 << 27) - 1 + (1 << 27)), Ev(x, t0 + 3 * (1 << 27) - 2)]
    tb.place(tb.stream_events(s, evs, ts_begin=t0))
    d = oracle.decode(tb.build())
    assert list(d["ts"]) == [ev.ts for ev in evs]
    assert list(d["ext"]) == [0, 0, 1, 0]


# -------------------------------------------------- ground-truth tallies
@pytest.mark.parametrize("name,over", [
    ("tiny", {}),
    ("tiny", dict(seed=7, total_calls=20_000, packet_bytes=256)),
    ("large", dict(total_calls=60_000, n_hosts=2, pids_per_host=2, tids_per_pid=4)),
    ("large", dict(total_calls=40_000, n_hosts=1, pids_per_host=1, tids_per_pid=2, p_long_gap=0.02,
                   p_sample=0.1, packet_bytes=512, seed=11)),
])
def test_tally_and_timeline_match_ground_truth(name, over):
    b, calls, _ev = tg.generate(tg.preset(name, **over), truth=True)
    r = oracle.run(b)
    assert r.code == oracle.OK
    rows, ivs = expected_from_truth(b, calls)
    assert rows_equal(r.rows, rows)
    assert intervals_equal(r.intervals, ivs)
    assert r.diag["pairs"] == len(calls)
    assert r.diag["unmatched_entries"] == r.diag["unmatched_exits"] == r.diag["mismatched_pairs"] == 0


def test_window_semantics():
    b, _c, _e = tg.generate(tg.preset("tiny", total_calls=5000))
    full = oracle.run(b)
    s, e = full.intervals["start_ns"], full.intervals["end_ns"]
    t0 = int(np.median(s))
    t1 = t0 + 200_000
    w = oracle.run(b, t0=t0, t1=t1)
    keep = (s < t1) & (e >= t0)
    assert intervals_equal(w.intervals, full.intervals[keep])
    assert rows_equal(w.rows, full.rows)


def test_stream_subset_matches_full_run():
    b, _c, _e = tg.generate(tg.preset("large", total_calls=40_000, n_hosts=2, pids_per_host=2, tids_per_pid=2))
    full = oracle.run(b)
    st = stream_table(b)
    sub = [1, 5, 6]
    part = oracle.run(b, streams=sub)
    keys = {(int(st[s][0]), int(st[s][1]), int(st[s][2])) for s in sub}
    mask = np.array([(r["host_id"], r["pid"], r["tid"]) in keys for r in full.rows])
    assert rows_equal(part.rows, full.rows[mask])
    assert intervals_equal(part.intervals, full.intervals[np.isin(full.intervals["stream_id"], sub)])


# ------------------------------------------------------------ brute force
def _trace_from_sequence(seq_by_stream, packet_bytes=256, payload=0):
    """seq: list of (kind, func) per stream; timestamps 10 ns apart; results alternate."""
    tb = TraceBuilder(packet_bytes=packet_bytes)
    h = tb.add_host("h")
    ids = [tb.add_call_func("f%d" % i) for i in range(2)]
    st = [tb.add_stream(h, 100, 100 + k) for k in range(len(seq_by_stream))]
    events_by_stream = []
    for k, seq in enumerate(seq_by_stream):
        evs, plain = [], []
        t = 1000 + 7 * k
        for j, (kind, func) in enumerate(seq):
            t += 10 + j
            res = (j % 3 == 1) * 5 if kind == EXIT else None
            cls = ids[func][1] if kind == ENTRY else ids[func][2]
            evs.append(Ev(cls, t, payload=b"\x11" * payload, result=res))
            plain.append((kind, func, t, res or 0))
        tb.place(tb.stream_events(st[k], evs, ts_begin=1000))
        events_by_stream.append(plain)
    return tb.build(), events_by_stream


def _brute_expect(trace, events_by_stream):
    st = stream_table(trace)
    flat, ivs = [], []
    diag = dict(pairs=0, mismatched_pairs=0, unmatched_entries=0, unmatched_exits=0)
    for sid, evs in enumerate(events_by_stream):
        pairs, mm, ue, ux = brute_force_stream(evs)
        diag["pairs"] += len(pairs)
        diag["mismatched_pairs"] += mm
        diag["unmatched_entries"] += ue
        diag["unmatched_exits"] += ux
        for (i, j, lvl) in pairs:
            dur = evs[j][2] - evs[i][2]
            err = 1 if evs[j][3] != 0 else 0
            flat.append((sid, evs[i][1], dur, err))
            ivs.append((evs[i][2], sid, i, evs[j][2], evs[i][1], min(lvl, 255), err))
    rows = tally_from_pairs(flat, st)
    ivs.sort(key=lambda v: (v[0], v[1], v[2]))
    arr = np.zeros(len(ivs), dtype=oracle.INTERVAL_DTYPE)
    for k, v in enumerate(ivs):
        arr[k] = (v[0], v[3], v[1], v[4], v[5], v[6])
    return rows, arr, diag


SYMBOLS = [(ENTRY, 0), (ENTRY, 1), (EXIT, 0), (EXIT, 1)]


def test_brute_force_all_short_sequences():
    n_checked = 0
    for length in range(1, 7):
        for seq in itertools.product(SYMBOLS, repeat=length):
            # two streams: the sequence and its reverse, so cross-stream keys are exercised
            trace, evs = _trace_from_sequence([list(seq), list(reversed(seq))])
            r = oracle.run(trace)
            assert r.code == oracle.OK
            rows, ivs, diag = _brute_expect(trace, evs)
            assert rows_equal(r.rows, rows), seq
            assert intervals_equal(r.intervals, ivs), seq
            for k, v in diag.items():
                assert r.diag[k] == v, (seq, k)
            n_checked += 1
    assert n_checked == sum(4 ** n for n in range(1, 7))


def test_brute_force_random_length_10_to_40():
    rng = random.Random(1234)
    for _ in range(400):
        length = rng.choice([10, 17, 40])
        # bias towards well-nested sequences with some noise
        seq, stack = [], []
        for _j in range(length):
            if stack and rng.random() < 0.45:
                f = stack.pop() if rng.random() > 0.1 else rng.randrange(2)
                seq.append((EXIT, f))
            elif rng.random() < 0.05:
                seq.append((EXIT, rng.randrange(2)))
            else:
                f = rng.randrange(2)
                stack.append(f)
                seq.append((ENTRY, f))
        trace, evs = _trace_from_sequence([seq], payload=rng.choice([0, 12, 40]))
        r = oracle.run(trace)
        rows, ivs, diag = _brute_expect(trace, evs)
        assert rows_equal(r.rows, rows)
        assert intervals_equal(r.intervals, ivs)
        for k, v in diag.items():
            assert r.diag[k] == v


# ----------------------------------------------------- hand-built cases
def _single_stream(calls_spec, packet_bytes=256, discarded_at=None, extra_events=None):
    """calls_spec: list of (kind, func_index, ts, result) already in stream order."""
    tb = TraceBuilder(packet_bytes=packet_bytes)
    h = tb.add_host("node0")
    ids = [tb.add_call_func("fn%d" % i, entry_fixed=8 * (i % 3)) for i in range(8)]
    s = tb.add_stream(h, 4242, 4243)
    evs = []
    for (kind, fi, ts, res) in calls_spec:
        evs.append(Ev(ids[fi][1] if kind == ENTRY else ids[fi][2], ts, result=res))
    tb.place(tb.stream_events(s, evs, ts_begin=calls_spec[0][2] if calls_spec else 0, discarded_at=discarded_at))
    return tb.build()


def _row_map(rows):
    return {int(r["func_id"]): (int(r["count"]), int(r["total_ns"]), int(r["min_ns"]), int(r["max_ns"]),
                                int(r["err_count"])) for r in rows}


def test_flat_calls():
    spec = [(ENTRY, 0, 100, None), (EXIT, 0, 150, 0), (ENTRY, 1, 200, None), (EXIT, 1, 230, 3),
            (ENTRY, 0, 300, None), (EXIT, 0, 310, 0)]
    r = oracle.run(_single_stream(spec))
    assert _row_map(r.rows) == {0: (2, 60, 10, 50, 0), 1: (1, 30, 30, 30, 1)}
    assert list(r.intervals["start_ns"]) == [100, 200, 300]
    assert list(r.intervals["level"]) == [0, 0, 0]
    assert list(r.intervals["flags"]) == [0, 1, 0]


def test_nested_depth_six_inclusive_time():
    spec = [(ENTRY, d, 1000 + 10 * d, None) for d in range(6)]
    spec += [(EXIT, d, 2000 - 10 * d, 0) for d in reversed(range(6))]
    r = oracle.run(_single_stream(spec))
    m = _row_map(r.rows)
    for d in range(6):
        dur = (2000 - 10 * d) - (1000 + 10 * d)
        assert m[d] == (1, dur, dur, dur, 0)
    # inclusive: every parent's time contains its child's
    assert all(m[d][1] > m[d + 1][1] for d in range(5))
    assert sorted(r.intervals["level"].tolist()) == list(range(6))


def test_layered_portable_over_vendor():
    # portable fn 0 calls vendor fns 1 and 2; vendor 2 calls vendor 3
    spec = [(ENTRY, 0, 10, None), (ENTRY, 1, 20, None), (EXIT, 1, 40, 0), (ENTRY, 2, 50, None),
            (ENTRY, 3, 55, None), (EXIT, 3, 70, 0), (EXIT, 2, 90, 0), (EXIT, 0, 100, 0)]
    r = oracle.run(_single_stream(spec))
    m = _row_map(r.rows)
    assert m == {0: (1, 90, 90, 90, 0), 1: (1, 20, 20, 20, 0), 2: (1, 40, 40, 40, 0), 3: (1, 15, 15, 15, 0)}
    lv = {int(i["func_id"]): int(i["level"]) for i in r.intervals}
    assert lv == {0: 0, 1: 1, 2: 1, 3: 2}


def test_dropped_entry_exit_and_mismatch():
    # exit of fn1 whose entry was dropped (unmatched exit), then fn2 whose exit was dropped
    # (unmatched entry at end), then mismatched: entry fn3 closed by exit fn4
    spec = [(EXIT, 1, 5, 0), (ENTRY, 3, 10, None), (EXIT, 4, 20, 0), (ENTRY, 0, 30, None), (EXIT, 0, 31, 0),
            (ENTRY, 2, 40, None)]
    r = oracle.run(_single_stream(spec, discarded_at={0: 2}))
    assert _row_map(r.rows) == {0: (1, 1, 1, 1, 0)}
    assert r.diag["unmatched_exits"] == 1
    assert r.diag["unmatched_entries"] == 1
    assert r.diag["mismatched_pairs"] == 1
    assert r.diag["discarded"] == 2
    assert r.diag["events"] == 6


def test_stream_crossing_many_packets():
    # one long outer call across many small packets, with many short children
    spec = [(ENTRY, 0, 1000, None)]
    t = 1000
    for k in range(300):
        spec.append((ENTRY, 1 + k % 5, t + 3, None))
        spec.append((EXIT, 1 + k % 5, t + 7, k % 50 == 0))
        t += 10
    spec.append((EXIT, 0, t + 1, 0))
    b = _single_stream(spec, packet_bytes=256)
    r = oracle.run(b)
    assert r.diag["packets"] > 20
    m = _row_map(r.rows)
    assert m[0] == (1, t + 1 - 1000, t + 1 - 1000, t + 1 - 1000, 0)
    assert sum(m[f][0] for f in range(1, 6)) == 300
    assert all(m[f][2] == 4 and m[f][3] == 4 for f in range(1, 6))
    assert sum(m[f][4] for f in range(1, 6)) == 6


def test_other_kinds_not_paired():
    tb = TraceBuilder(packet_bytes=256)
    h = tb.add_host("h")
    f, e, x = tb.add_call_func("f")
    fs = tb.add_func("sample")
    cs = tb.add_class(fs, SAMPLE, 8)
    cb = tb.add_class(fs, DEV_BEGIN, 8, cmd_off=0)
    s = tb.add_stream(h, 1, 1)
    tb.place(tb.stream_events(s, [Ev(e, 10), Ev(cs, 12), Ev(cb, 13, cmd=99), Ev(x, 20, result=0)], ts_begin=5))
    r = oracle.run(tb.build())
    assert r.diag["other_events"] == 2 and r.diag["pairs"] == 1
    assert int(r.rows[0]["total_ns"]) == 10


# ------------------------------------------------------- invariants
@pytest.mark.parametrize("seed", [3, 4])
def test_invariants_with_drops(seed):
    cfg = tg.preset("large", total_calls=50_000, n_hosts=1, pids_per_host=2, tids_per_pid=3, p_drop=0.003,
                    p_sample=0.05, seed=seed, packet_bytes=1024)
    b, calls, _ev = tg.generate(cfg, truth=True)
    r = oracle.run(b)
    d = r.diag
    assert d["unmatched_entries"] + d["unmatched_exits"] + d["mismatched_pairs"] > 0
    assert d["events"] == 2 * (d["pairs"] + d["mismatched_pairs"]) + d["unmatched_entries"] + \
        d["unmatched_exits"] + d["other_events"]
    dropped = int(((calls["flags"] & 2) > 0).sum() + ((calls["flags"] & 4) > 0).sum())
    assert d["discarded"] >= dropped  # samples can be dropped too
    assert int(r.rows["count"].sum()) == d["pairs"] == len(r.intervals)
    durs = (r.intervals["end_ns"] - r.intervals["start_ns"]).astype(np.uint64)
    assert int(r.rows["total_ns"].astype(object).sum()) == int(durs.astype(object).sum())
    assert np.all(r.rows["min_ns"] * r.rows["count"] <= r.rows["total_ns"])
    assert np.all(r.rows["total_ns"] <= r.rows["max_ns"] * r.rows["count"])
    s = r.intervals["start_ns"]
    assert np.all(s[1:] >= s[:-1])
    # nesting well-formed: per stream, a level-L+1 interval lies inside the latest level-L interval
    for sid in np.unique(r.intervals["stream_id"])[:3]:
        iv = r.intervals[r.intervals["stream_id"] == sid]
        open_by_level = {}
        for row in iv:
            lvl = int(row["level"])
            if lvl > 0 and (lvl - 1) in open_by_level:
                ps, pe = open_by_level[lvl - 1]
                if ps <= row["start_ns"] <= pe:
                    assert row["end_ns"] <= pe
            open_by_level[lvl] = (row["start_ns"], row["end_ns"])


# ----------------------------------------------------------- errors
def _good_builder():
    tb = TraceBuilder(packet_bytes=256)
    h = tb.add_host("h")
    f, e, x = tb.add_call_func("f")
    s0 = tb.add_stream(h, 1, 1)
    s1 = tb.add_stream(h, 1, 2)
    return tb, e, x, s0, s1


def _expect(trace, code, loc=None):
    r = oracle.run(trace)
    assert r.code == code
    if loc is not None:
        assert r.loc == loc
    return r


def test_error_file_level():
    tb, e, x, s0, s1 = _good_builder()
    tb.raw_packet(s0, 0, [tb.encode_event(e, 1), tb.encode_event(x, 2)])
    good = tb.build()
    assert oracle.run(good).code == oracle.OK
    _expect(good[:100], oracle.E_TRUNCATED)
    _expect(b"XXXX" + good[4:], oracle.E_FORMAT)
    _expect(tb.build({4: ("<H", 2)}), oracle.E_FORMAT)                 # version
    _expect(tb.build({8: ("<I", 300)}), oracle.E_FORMAT)               # packet size not a power of two
    _expect(tb.build({32: ("<Q", 5)}), oracle.E_TRUNCATED)             # more packets than bytes
    _expect(tb.build({88: ("<Q", 300)}), oracle.E_FORMAT)              # packets not 256-aligned
    _expect(good[:-10], oracle.E_TRUNCATED)


def test_error_tables():
    tb, e, x, s0, s1 = _good_builder()
    tb.classes[e].kind = 9
    _expect(tb.build(), oracle.E_FORMAT)
    tb, e, x, s0, s1 = _good_builder()
    tb.classes[x].fixed = 6
    _expect(tb.build(), oracle.E_FORMAT)
    tb, e, x, s0, s1 = _good_builder()
    tb.classes[x].result_off = 4  # beyond fixed part
    _expect(tb.build(), oracle.E_FORMAT)
    tb, e, x, s0, s1 = _good_builder()
    tb.streams[s1] = (7, 1, 2, 0)   # host out of range
    _expect(tb.build(), oracle.E_FORMAT)


def test_error_packet_headers_precede_content():
    tb, e, x, s0, s1 = _good_builder()
    tb.raw_packet(s0, 0, [tb.encode_event(e, 1, raw_tsw=0x10000000)])  # content error in packet 0
    tb.raw_packet(s1, 0, [tb.encode_event(e, 1)], magic=0xDEAD)           # header error in packet 1
    _expect(tb.build(), oracle.E_FORMAT, (1, 1, 0))


@pytest.mark.parametrize("case,code,event", [
    ("tsw_high_bits", oracle.E_FORMAT, 1),
    ("bad_class", oracle.E_FORMAT, 1),
    ("ext_with_delta", oracle.E_FORMAT, 1),
    ("event_overruns", oracle.E_TRUNCATED, 1),
    ("header_overruns", oracle.E_TRUNCATED, 1),
    ("count_mismatch", oracle.E_FORMAT, 2),
])
def test_error_content(case, code, event):
    tb, e, x, s0, s1 = _good_builder()
    tb.raw_packet(s0, 0, [tb.encode_event(e, 1), tb.encode_event(x, 2)])
    good = tb.encode_event(e, 3)
    if case == "tsw_high_bits":
        evs = [good, tb.encode_event(x, raw_tsw=0x20000005)]
        tb.raw_packet(s1, 0, evs)
    elif case == "bad_class":
        evs = [good, struct.pack("<IHH", 1, 77, 0)]
        tb.raw_packet(s1, 0, evs)
    elif case == "ext_with_delta":
        evs = [good, tb.encode_event(x, raw_tsw=(1 << 27) | 4, ext_ts=50)]
        tb.raw_packet(s1, 0, evs)
    elif case == "event_overruns":
        evs = [good, tb.encode_event(x, 1, payload=b"\x00" * 8)]
        tb.raw_packet(s1, 0, evs, content_bytes=len(good) + 12)
    elif case == "header_overruns":
        evs = [good, b"\x01\x00\x00\x00"]
        tb.raw_packet(s1, 0, evs, n_events=1)
    elif case == "count_mismatch":
        evs = [good, tb.encode_event(x, 1)]
        tb.raw_packet(s1, 0, evs, n_events=1)
    _expect(tb.build(), code, (2, 1, event))


def test_error_seq_and_header_fields():
    tb, e, x, s0, s1 = _good_builder()
    tb.raw_packet(s0, 0, [tb.encode_event(e, 1)], seq=5)
    tb.raw_packet(s0, 0, [tb.encode_event(x, 1)], seq=5)
    _expect(tb.build(), oracle.E_FORMAT, (1, 1, 0))
    tb, e, x, s0, s1 = _good_builder()
    tb.raw_packet(9, 0, [tb.encode_event(e, 1)])
    _expect(tb.build(), oracle.E_FORMAT, (1, 0, 0))
    tb, e, x, s0, s1 = _good_builder()
    tb.raw_packet(s0, 0, [tb.encode_event(e, 1)], content_bytes=6)
    _expect(tb.build(), oracle.E_FORMAT, (1, 0, 0))
    tb, e, x, s0, s1 = _good_builder()
    tb.raw_packet(s0, 0, [tb.encode_event(e, 1)], n_events=2)
    _expect(tb.build(), oracle.E_FORMAT, (1, 0, 0))


# ------------------------------------------------ device-activity pairing
def test_device_pairing_handbuilt_cases():
    from tests import _device_trace as dt
    b, ids = dt.build()
    r = oracle.run(b)
    assert r.code == oracle.OK
    assert r.dev_diag == dt.EXPECTED_DEV_DIAG
    assert dt.as_tuples(r.dev_rows) == dt.expected_dev_rows(ids)
    dev = r.intervals[(r.intervals["flags"] & oracle.IV_DEVICE) != 0]
    assert dt.as_tuples(dev) == dt.expected_dev_intervals(ids)
    # the host calls themselves are ordinary intervals; device events are other events
    assert r.diag["pairs"] == 9 and r.diag["other_events"] == 17
    assert len(r.intervals) == 9 + 3
    # the host tally has no device rows
    assert set(int(x) for x in r.rows["pid"]) == {7}


@pytest.mark.parametrize("over", [
    dict(total_calls=20_000, n_hosts=1, pids_per_host=2, tids_per_pid=2, n_device_streams=3),
    dict(total_calls=30_000, n_hosts=2, pids_per_host=2, tids_per_pid=2, n_device_streams=5, packet_bytes=1024,
         p_ext=0.01, seed=5),
])
def test_device_pairing_matches_ground_truth(over):
    b, calls, _ev = tg.generate(tg.preset("device", **over), truth=True)
    r = oracle.run(b)
    assert r.code == oracle.OK
    rows, ivs, diag = expected_device_from_truth(b, calls)
    assert r.dev_diag == diag
    assert rows_equal(r.dev_rows, rows)
    # whole timeline = host calls and device intervals merged by (start, stream, position)
    host_rows, host_ivs = expected_from_truth(b, calls)
    assert rows_equal(r.rows, host_rows)
    host_seq = np.flatnonzero((calls["flags"] & 8) == 0)
    dev_seq = np.flatnonzero((calls["flags"] & 8) != 0)
    host_ivs_seq = host_seq[np.lexsort((host_seq, calls["stream_id"][host_seq], calls["start_ns"][host_seq]))]
    dev_ivs_seq = dev_seq[np.lexsort((dev_seq, calls["stream_id"][dev_seq], calls["start_ns"][dev_seq]))]
    merged = merge_timelines(host_ivs, host_ivs_seq, ivs, dev_ivs_seq)
    assert intervals_equal(r.intervals, merged)


@pytest.mark.parametrize("seed", [6, 7])
def test_device_pairing_with_drops_matches_ground_truth(seed):
    cfg = tg.preset("device", total_calls=30_000, n_hosts=1, pids_per_host=2, tids_per_pid=3, n_device_streams=4,
                    p_drop=0.01, seed=seed, packet_bytes=1024)
    b, calls, _ev = tg.generate(cfg, truth=True)
    r = oracle.run(b)
    rows, ivs, diag = expected_device_from_truth(b, calls)
    assert diag["dev_unpaired"] > 0 and diag["dev_unjoined"] > 0 and diag["host_unjoined"] > 0
    assert r.dev_diag == diag
    assert rows_equal(r.dev_rows, rows)
    assert intervals_equal(r.intervals[(r.intervals["flags"] & oracle.IV_DEVICE) != 0], ivs)


def test_device_invariants():
    cfg = tg.preset("device", total_calls=40_000, n_hosts=1, pids_per_host=2, tids_per_pid=2, n_device_streams=6,
                    p_drop=0.005, seed=9, packet_bytes=512)
    b, _c, _e = tg.generate(cfg)
    r = oracle.run(b)
    dd = r.dev_diag
    assert dd["dev_events"] == 2 * dd["dev_pairs"] + dd["dev_unpaired"]
    assert dd["dev_pairs"] == dd["dev_intervals"] + dd["dev_unjoined"] + dd["dev_ambiguous"]
    dev = r.intervals[(r.intervals["flags"] & oracle.IV_DEVICE) != 0]
    assert int(r.dev_rows["count"].sum()) == dd["dev_intervals"] == len(dev)
    durs = (dev["end_ns"] - dev["start_ns"]).astype(object)
    assert int(r.dev_rows["total_ns"].astype(object).sum()) == int(durs.sum())
    assert np.all(dev["level"] == 0) and np.all(r.dev_rows["err_count"] == 0)
    s = r.intervals["start_ns"]
    assert np.all(s[1:] >= s[:-1])
    # device events are the other events of this model (no samples)
    assert r.diag["other_events"] == dd["dev_events"]


def test_device_window_keeps_overlapping_device_intervals():
    from tests import _device_trace as dt
    b, ids = dt.build()
    full = oracle.run(b)
    w = oracle.run(b, t0=dt.T0 + 150, t1=dt.T0 + 131)
    keep = (full.intervals["start_ns"] < dt.T0 + 131) & (full.intervals["end_ns"] >= dt.T0 + 150)
    assert intervals_equal(w.intervals, full.intervals[keep])
    assert dt.as_tuples(w.intervals[(w.intervals["flags"] & 4) != 0])[0][:2] == (dt.T0 + 100, dt.T0 + 150)


# --------------------------------------------------------- per-CPU buffers
def _iv_key(ivs):
    return sorted((int(v["start_ns"]), int(v["end_ns"]), int(v["func_id"]), int(v["level"]), int(v["flags"]))
                  for v in ivs)


@pytest.mark.parametrize("over,n_cpus", [
    (dict(total_calls=20_000, n_hosts=2, pids_per_host=2, tids_per_pid=2, seed=3, p_drop=0.005), 3),
    (dict(total_calls=15_000, n_hosts=1, pids_per_host=2, tids_per_pid=4, seed=4, p_ext=0.02, packet_bytes=512), 2),
])
def test_per_cpu_buffers_give_the_per_thread_results(over, n_cpus):
    """The same calls written per thread and per CPU (threads migrating between
    CPUs) give the same tally, the same pairing diagnostics and the same
    intervals up to the stream they belong to."""
    from tests._percpu import to_per_cpu
    b, _c, _e = tg.generate(tg.preset("large", **over))
    pc = to_per_cpu(b, n_cpus=n_cpus, seed=over["seed"])
    r1, r2 = oracle.run(b), oracle.run(pc)
    assert r2.code == oracle.OK
    assert rows_equal(r1.rows, r2.rows)
    for k in ("events", "pairs", "unmatched_entries", "unmatched_exits", "mismatched_pairs", "other_events"):
        assert r1.diag[k] == r2.diag[k], k
    assert _iv_key(r1.intervals) == _iv_key(r2.intervals)
    s = r2.intervals["start_ns"]
    assert np.all(s[1:] >= s[:-1])


def test_per_cpu_thread_migrates_inside_a_call():
    """Thread (pid 5, tid 7) enters f on CPU 0 and g inside it, then migrates: g and f exit on CPU 1.
    Thread (5, 8) interleaves on CPU 0 with its own call.  Written out by hand."""
    tb = TraceBuilder(packet_bytes=256)
    h = tb.add_host("h")
    f, ef, xf = tb.add_call_func("f")
    g, eg, xg = tb.add_call_func("g")
    c0, c1 = tb.add_stream(h, 0, 0, 2), tb.add_stream(h, 0, 1, 2)
    A, B = (5, 7), (5, 8)
    cpu0 = [Ev(ef, 100, ctx=A), Ev(ef, 105, ctx=B), Ev(eg, 110, ctx=A), Ev(xf, 130, result=3, ctx=B)]
    cpu1 = [Ev(xg, 140, result=0, ctx=A), Ev(xf, 170, result=0, ctx=A)]
    tb.place(tb.stream_events(c0, cpu0, ts_begin=100))
    tb.place(tb.stream_events(c1, cpu1, ts_begin=100))
    r = oracle.run(tb.build())
    assert r.code == oracle.OK and r.diag["pairs"] == 3
    rows = [tuple(int(v) for v in x) for x in r.rows.tolist()]
    assert rows == [(0, 5, 7, f, 1, 70, 70, 70, 0), (0, 5, 7, g, 1, 30, 30, 30, 0), (0, 5, 8, f, 1, 25, 25, 25, 1)]
    ivs = [tuple(int(v) for v in x) for x in r.intervals.tolist()]
    # (start, end, stream of the entry, func, level, flags), by start
    assert ivs == [(100, 170, c0, f, 0, 0), (105, 130, c0, f, 0, 1), (110, 140, c0, g, 1, 0)]


def test_per_cpu_header_truncated():
    tb = TraceBuilder(packet_bytes=256)
    h = tb.add_host("h")
    f, e, x = tb.add_call_func("f")
    c0 = tb.add_stream(h, 0, 0, 2)
    ok = tb.encode_event(e, 1, ctx=(1, 1))
    tb.raw_packet(c0, 0, [ok, ok[:12]], n_events=2)  # the second event's 16-byte header is cut
    r = oracle.run(tb.build())
    assert r.code == oracle.E_TRUNCATED and r.loc == (2, 0, 1)


# ------------------------------------------------------------ self time
def test_self_time_layered_worked_case():
    """The layering of Sec. 4.3 by hand: hipDeviceSynchronize [0, 100] waits in
    two zeEventHostSynchronize calls [10, 40] and [50, 95]; the first of them
    makes a leaf call [12, 20].  A call's self time loses only its direct
    children: hip 100 - 30 - 45 = 25, ze 30 - 8 = 22 and 45, the leaf 8."""
    tb = TraceBuilder(packet_bytes=256)
    h = tb.add_host("h")
    hip, eh, xh = tb.add_call_func("hipDeviceSynchronize", layer=0)
    ze, ez, xz = tb.add_call_func("zeEventHostSynchronize", layer=1)
    lf, el, xl = tb.add_call_func("leaf", layer=1)
    s = tb.add_stream(h, 1, 1)
    evs = [Ev(eh, 1000), Ev(ez, 1010), Ev(el, 1012), Ev(xl, 1020, result=0), Ev(xz, 1040, result=0),
           Ev(ez, 1050), Ev(xz, 1095, result=0), Ev(xh, 1100, result=2)]
    tb.place(tb.stream_events(s, evs, ts_begin=1000))
    r = oracle.run(tb.build())
    assert r.code == oracle.OK
    got = {int(x["func_id"]): tuple(int(x[k]) for k in ("count", "total_ns", "min_ns", "max_ns", "err_count"))
           for x in r.self_rows}
    assert got == {hip: (1, 25, 25, 25, 1), ze: (2, 22 + 45, 22, 45, 0), lf: (1, 8, 8, 8, 0)}
    incl = {int(x["func_id"]): int(x["total_ns"]) for x in r.rows}
    assert incl == {hip: 100, ze: 75, lf: 8}


def test_self_time_invalid_parents_take_nothing():
    """A mismatched call (entry f, exit g) and a call never closed have no
    duration: the paired calls directly inside them take nothing off any
    call, and the mismatched call takes nothing off its own parent."""
    tb = TraceBuilder(packet_bytes=256)
    h = tb.add_host("h")
    f, ef, xf = tb.add_call_func("f")
    g, eg, xg = tb.add_call_func("g")
    c, ec, xc = tb.add_call_func("c")
    s = tb.add_stream(h, 1, 1)
    evs = [Ev(ef, 100),                                   # f [100, 200]
           Ev(eg, 110), Ev(ec, 120), Ev(xc, 130, result=0), Ev(xf, 140, result=0),  # g..f mismatched, c inside
           Ev(ec, 150), Ev(xc, 155, result=0),            # c directly in f: 5
           Ev(xf, 200, result=0),
           Ev(eg, 300), Ev(ec, 310), Ev(xc, 330, result=0)]  # g never closed, c inside it
    tb.place(tb.stream_events(s, evs, ts_begin=100))
    r = oracle.run(tb.build())
    assert r.diag["mismatched_pairs"] == 1 and r.diag["unmatched_entries"] == 1
    got = {int(x["func_id"]): (int(x["count"]), int(x["total_ns"])) for x in r.self_rows}
    assert got == {f: (1, 100 - 5), c: (3, 10 + 5 + 20)}


@pytest.mark.parametrize("over", [
    dict(total_calls=20_000, seed=11),
    dict(total_calls=20_000, seed=12, n_hosts=2, pids_per_host=2, tids_per_pid=2, packet_bytes=512, p_ext=0.02),
])
def test_self_time_from_truth(over):
    b, calls, _e = tg.generate(tg.preset("large", p_drop=0.0, **over), truth=True)
    r = oracle.run(b)
    from tests._util import self_from_truth
    exp = self_from_truth(b, calls)
    assert rows_equal(r.self_rows, exp)
    # keys, counts and error counts are the tally's
    for k in ("host_id", "pid", "tid", "func_id", "count", "err_count"):
        assert np.array_equal(r.self_rows[k], r.rows[k]), k
    # every call's time is counted once: as self time of itself or of its ancestors
    lvl0 = r.intervals[r.intervals["level"] == 0]
    total0 = int((lvl0["end_ns"] - lvl0["start_ns"]).astype(np.uint64).sum(dtype=np.uint64))
    assert int(r.self_rows["total_ns"].sum(dtype=np.uint64)) == total0


def test_self_time_flat_calls_equal_inclusive():
    b, _c, _e = tg.generate(tg.preset("tiny", seed=5))
    r = oracle.run(b)
    if int(r.intervals["level"].max()) == 0:
        assert rows_equal(r.self_rows, r.rows)
    assert np.all(r.self_rows["total_ns"] <= r.rows["total_ns"])


def _brute_self_rows(trace, events_by_stream):
    from tests._util import brute_force_self
    st = stream_table(trace)
    flat = []
    for sid, evs in enumerate(events_by_stream):
        for (i, j, _lvl, self_ns) in brute_force_self(evs):
            flat.append((sid, evs[i][1], self_ns, 1 if evs[j][3] != 0 else 0))
    return tally_from_pairs(flat, st)


def test_self_time_brute_force_short_sequences():
    for length in range(1, 7):
        for seq in itertools.product(SYMBOLS, repeat=length):
            trace, evs = _trace_from_sequence([list(seq), list(reversed(seq))])
            r = oracle.run(trace)
            assert rows_equal(r.self_rows, _brute_self_rows(trace, evs)), seq


def test_self_time_brute_force_random():
    rng = random.Random(77)
    for _ in range(300):
        length = rng.choice([12, 25, 60])
        seq, stack = [], []
        for _j in range(length):
            if stack and rng.random() < 0.45:
                f = stack.pop() if rng.random() > 0.1 else rng.randrange(2)
                seq.append((EXIT, f))
            elif rng.random() < 0.05:
                seq.append((EXIT, rng.randrange(2)))
            else:
                f = rng.randrange(2)
                stack.append(f)
                seq.append((ENTRY, f))
        trace, evs = _trace_from_sequence([seq])
        r = oracle.run(trace)
        assert rows_equal(r.self_rows, _brute_self_rows(trace, evs))


def test_self_time_per_cpu_equals_per_thread():
    from tests._percpu import to_per_cpu
    b, _c, _e = tg.generate(tg.preset("large", total_calls=15_000, n_hosts=1, pids_per_host=2, tids_per_pid=3,
                                      seed=21, p_drop=0.01))
    pc = to_per_cpu(b, n_cpus=3, seed=21)
    assert rows_equal(oracle.run(b).self_rows, oracle.run(pc).self_rows)


@pytest.mark.parametrize("over", [
    dict(total_calls=20_000, n_hosts=2, pids_per_host=2, tids_per_pid=3, n_cpus=4, slice_ns=30_000.0, seed=41,
         p_drop=0.005),
    dict(total_calls=15_000, n_hosts=1, pids_per_host=1, tids_per_pid=4, n_cpus=2, slice_ns=5_000.0, seed=42,
         p_ext=0.02, packet_bytes=1024),
])
def test_generator_per_cpu_mode_writes_the_same_calls(over):
    """The generator's per-CPU buffers (threads scheduled onto CPUs in time
    slices) carry the same calls as its per-thread streams with the same seed:
    the oracle gives the same tally, self time, diagnostics and intervals."""
    per_cpu = tg.generate(tg.preset("large", **over))[0]
    per_thread = tg.generate(tg.preset("large", **dict(over, n_cpus=0)))[0]
    a, b = oracle.run(per_thread), oracle.run(per_cpu)
    assert b.code == oracle.OK
    st = stream_table(per_cpu)
    assert np.all(st[:, 3] == 2) and len(st) == over["n_hosts"] * over["n_cpus"]
    assert rows_equal(a.rows, b.rows) and rows_equal(a.self_rows, b.self_rows)
    for k in ("events", "pairs", "unmatched_entries", "unmatched_exits", "mismatched_pairs", "other_events",
              "discarded"):
        assert a.diag[k] == b.diag[k], k
    assert _iv_key(a.intervals) == _iv_key(b.intervals)
    ev = oracle.decode(per_cpu)
    # threads migrate: some thread has events in more than one buffer
    sids = {}
    for t, s in zip(ev["vtid"].tolist(), ev["stream_id"].tolist()):
        sids.setdefault(t, set()).add(s)
    assert max(len(v) for v in sids.values()) > 1
