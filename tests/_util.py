"""Test helpers: independent expectations built from generator ground truth,
a brute-force depth-based matcher, and small header readers.

Nothing here is shared with the oracle or the CUDA library: the expectations
are restated from the definitions (group-by over ground-truth calls; the
clamped-depth formulation of entry/exit pairing) so that they can catch a
mistake in either implementation.
"""
from __future__ import annotations

import struct
from collections import defaultdict

import numpy as np

ENTRY, EXIT = 0, 1
U64 = (1 << 64) - 1

ROW_DTYPE = np.dtype([("host_id", "<u4"), ("pid", "<u4"), ("tid", "<u4"), ("func_id", "<u4"),
                      ("count", "<u8"), ("total_ns", "<u8"), ("min_ns", "<u8"), ("max_ns", "<u8"),
                      ("err_count", "<u8")])
INTERVAL_DTYPE = np.dtype([("start_ns", "<u8"), ("end_ns", "<u8"), ("stream_id", "<u4"),
                           ("func_id", "<u2"), ("level", "u1"), ("flags", "u1")])


def stream_table(trace) -> np.ndarray:
    """(n_streams, 4) array of host_id, pid, tid, flags read from the file header."""
    b = bytes(trace[:128]) if isinstance(trace, np.ndarray) else trace[:128]
    n_streams = struct.unpack_from("<I", b, 12)[0]
    off = struct.unpack_from("<Q", b, 40)[0]
    raw = np.asarray(trace[off: off + 16 * n_streams]) if isinstance(trace, np.ndarray) else \
        np.frombuffer(trace[off: off + 16 * n_streams], dtype=np.uint8)
    return np.frombuffer(raw.tobytes(), dtype="<u4").reshape(n_streams, 4)


def expected_from_truth(trace, calls: np.ndarray):
    """Tally rows and timeline implied by ground-truth calls of a drop-free trace."""
    st = stream_table(trace)
    host_calls = calls[(calls["flags"] & 8) == 0]
    dur = (host_calls["end_ns"] - host_calls["start_ns"]).astype(np.uint64)
    err = (host_calls["flags"] & 1).astype(np.uint64)
    sid = host_calls["stream_id"].astype(np.int64)
    keys = np.stack([st[sid, 0], st[sid, 1], st[sid, 2], host_calls["func_id"].astype(np.uint32)], axis=1)
    order = np.lexsort((keys[:, 3], keys[:, 2], keys[:, 1], keys[:, 0]))
    keys_s = keys[order]
    new = np.ones(len(order), dtype=bool)
    if len(order) > 1:
        new[1:] = np.any(keys_s[1:] != keys_s[:-1], axis=1)
    starts = np.flatnonzero(new)
    rows = np.zeros(len(starts), dtype=ROW_DTYPE)
    rows["host_id"], rows["pid"], rows["tid"], rows["func_id"] = (keys_s[starts, i] for i in range(4))
    d_s, e_s = dur[order], err[order]
    rows["count"] = np.diff(np.append(starts, len(order)))
    rows["total_ns"] = np.add.reduceat(d_s, starts) if len(order) else []
    rows["min_ns"] = np.minimum.reduceat(d_s, starts) if len(order) else []
    rows["max_ns"] = np.maximum.reduceat(d_s, starts) if len(order) else []
    rows["err_count"] = np.add.reduceat(e_s, starts) if len(order) else []
    # timeline: (start, stream, entry order); calls are recorded in entry order per stream
    ivs = np.zeros(len(host_calls), dtype=INTERVAL_DTYPE)
    ivs["start_ns"] = host_calls["start_ns"]
    ivs["end_ns"] = host_calls["end_ns"]
    ivs["stream_id"] = host_calls["stream_id"]
    ivs["func_id"] = host_calls["func_id"]
    ivs["level"] = host_calls["level"]
    ivs["flags"] = host_calls["flags"] & 1
    seq = np.arange(len(host_calls))
    t_order = np.lexsort((seq, host_calls["stream_id"], host_calls["start_ns"]))
    return rows, ivs[t_order]


def brute_force_stream(events):
    """Pairs one stream's events by the clamped-depth definition, by brute force.

    events: list of (kind, func, ts, result).  The running sum S of +1 (entry)
    and -1 (exit) is clamped by its prefix minimum, so the depth before event j
    is S_{j-1} - min(S_0..S_{j-1}).  An entry at depth L pairs with the first
    later exit whose depth before it is L + 1; an exit seen at depth 0 is
    unmatched.  O(n^2) on purpose.
    """
    n = len(events)
    s = [0]
    for (k, _f, _t, _r) in events:
        s.append(s[-1] + (1 if k == ENTRY else (-1 if k == EXIT else 0)))
    pre = []
    for j in range(n):
        pre.append(s[j] - min(s[: j + 1]))
    pairs, mismatched, un_entry, un_exit = [], 0, 0, 0
    for j in range(n):
        if events[j][0] == EXIT and pre[j] == 0:
            un_exit += 1
    for i in range(n):
        if events[i][0] != ENTRY:
            continue
        match = None
        for j in range(i + 1, n):
            if events[j][0] == EXIT and pre[j] - 1 == pre[i]:
                match = j
                break
        if match is None:
            un_entry += 1
        elif events[match][1] != events[i][1]:
            mismatched += 1
        else:
            pairs.append((i, match, pre[i]))
    return pairs, mismatched, un_entry, un_exit


def brute_force_self(events):
    """Self time of each pair of brute_force_stream, by brute force.

    Returns (i, j, level, self) per pair: the pair's duration less the
    durations of the pairs whose direct parent it is.  The direct parent of an
    entry at depth L > 0 is the last earlier entry at depth L - 1 (the one
    open at that depth when it is pushed); it takes the child's duration only
    when it is itself a pair.  Depths by the clamped running sum, as in
    brute_force_stream; O(n^2) on purpose.
    """
    pairs, _mm, _ue, _ux = brute_force_stream(events)
    n = len(events)
    s = [0]
    for (k, _f, _t, _r) in events:
        s.append(s[-1] + (1 if k == ENTRY else (-1 if k == EXIT else 0)))
    pre = [s[j] - min(s[: j + 1]) for j in range(n)]
    paired = {i for (i, _j, _l) in pairs}
    child = defaultdict(int)
    for (i, j, lvl) in pairs:
        if lvl == 0:
            continue
        k = max(k for k in range(i) if events[k][0] == ENTRY and pre[k] == lvl - 1)
        if k in paired:
            child[k] += (events[j][2] - events[i][2]) & U64
    return [(i, j, lvl, ((events[j][2] - events[i][2]) - child[i]) & U64) for (i, j, lvl) in pairs]


def self_from_truth(trace, calls: np.ndarray):
    """Self-time rows implied by the ground-truth calls of a drop-free trace: per
    stream, in entry order, a call's parent is the last earlier call one level up."""
    st = stream_table(trace)
    host = calls[(calls["flags"] & 8) == 0]
    out = []
    for sid in np.unique(host["stream_id"]):
        cs = host[host["stream_id"] == sid]
        dur = [(int(c["end_ns"]) - int(c["start_ns"])) & U64 for c in cs]
        child = [0] * len(cs)
        last_at = {}
        for k, c in enumerate(cs):
            lvl = int(c["level"])
            if lvl > 0:
                child[last_at[lvl - 1]] += dur[k]
            last_at[lvl] = k
        for k, c in enumerate(cs):
            out.append((int(sid), int(c["func_id"]), (dur[k] - child[k]) & U64, int(c["flags"]) & 1))
    return tally_from_pairs(out, st)


def tally_from_pairs(pairs_by_stream, st):
    """Group-by over (host, pid, tid, func) of (stream, func, dur, err) tuples."""
    acc = defaultdict(lambda: [0, 0, U64, 0, 0])
    for (sid, func, dur, err) in pairs_by_stream:
        h, p, t = int(st[sid][0]), int(st[sid][1]), int(st[sid][2])
        a = acc[(h, p, t, func)]
        a[0] += 1
        a[1] = (a[1] + dur) & U64
        a[2] = min(a[2], dur)
        a[3] = max(a[3], dur)
        a[4] += err
    keys = sorted(acc)
    rows = np.zeros(len(keys), dtype=ROW_DTYPE)
    for i, k in enumerate(keys):
        rows[i] = (*k, *acc[k])
    return rows


def rows_equal(a, b) -> bool:
    return len(a) == len(b) and all(np.array_equal(a[f], b[f]) for f in ROW_DTYPE.names)


def intervals_equal(a, b) -> bool:
    return len(a) == len(b) and all(np.array_equal(a[f], b[f]) for f in INTERVAL_DTYPE.names)


def expected_device_from_truth(trace, calls: np.ndarray):
    """Device tally rows, device intervals (timeline order) and the device
    diagnostics implied by the generator's ground truth of a device-model
    trace, drops included.

    In that model every host call issues one command with a unique id, so a
    truth record of a device command (flag 8) is a device interval exactly
    when neither its DEV_BEGIN (flag 2) nor its DEV_END (flag 4) nor the
    issuing call's ENTRY (flag 16) was dropped.
    """
    st = stream_table(trace)
    dev_all = calls[(calls["flags"] & 8) != 0]
    host = calls[(calls["flags"] & 8) == 0]
    seq = np.flatnonzero((calls["flags"] & 8) != 0)  # stream-major truth order = stream order
    paired = (dev_all["flags"] & 6) == 0
    joined = paired & ((dev_all["flags"] & 16) == 0)
    dev = dev_all[joined]
    dev_seq = seq[joined]
    dev_events = 2 * len(dev_all) - int(((dev_all["flags"] & 2) != 0).sum()) - int(((dev_all["flags"] & 4) != 0).sum())
    host_cmd_entries = int(((host["flags"] & 2) == 0).sum())
    diag = dict(dev_events=dev_events, dev_pairs=int(paired.sum()), dev_intervals=int(joined.sum()),
                dev_unpaired=dev_events - 2 * int(paired.sum()), dev_unjoined=int((paired & ~joined).sum()),
                dev_ambiguous=0, host_cmd_entries=host_cmd_entries,
                host_unjoined=host_cmd_entries - int(joined.sum()))
    acc = defaultdict(lambda: [0, 0, U64, 0, 0])
    for r in dev:
        sid = int(r["stream_id"])
        d = int(r["end_ns"]) - int(r["start_ns"])
        a = acc[(int(st[sid][0]), int(st[sid][1]), int(st[sid][2]), int(r["func_id"]))]
        a[0] += 1
        a[1] += d
        a[2] = min(a[2], d)
        a[3] = max(a[3], d)
    keys = sorted(acc)
    rows = np.zeros(len(keys), dtype=ROW_DTYPE)
    for i, k in enumerate(keys):
        rows[i] = (*k, *acc[k])
    ivs = np.zeros(len(dev), dtype=INTERVAL_DTYPE)
    ivs["start_ns"], ivs["end_ns"] = dev["start_ns"], dev["end_ns"]
    ivs["stream_id"], ivs["func_id"] = dev["stream_id"], dev["func_id"]
    ivs["flags"] = 4
    order = np.lexsort((dev_seq, dev["stream_id"], dev["start_ns"]))
    return rows, ivs[order], diag


def merge_timelines(a: np.ndarray, a_seq: np.ndarray, b: np.ndarray, b_seq: np.ndarray) -> np.ndarray:
    """Two timelines over disjoint streams merged in (start, stream, position) order."""
    allv = np.concatenate([a, b])
    seq = np.concatenate([a_seq, b_seq])
    return allv[np.lexsort((seq, allv["stream_id"], allv["start_ns"]))]
