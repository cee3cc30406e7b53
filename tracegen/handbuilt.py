"""Hand-built THPT traces for pins and edge cases (input writer only).

Two levels:

* ``TraceBuilder.stream_events`` takes a stream's events with absolute
  timestamps and packs them into packets the way a tracer would (delta
  encoding, EXT when a delta needs more than 27 bits or is negative, a new
  packet when the next event does not fit).
* ``TraceBuilder.raw_packet`` writes one packet from explicit header fields
  and pre-encoded event byte strings, for malformed-input cases.

Layout (little-endian): 128-byte file header; stream rows {host_id, pid, tid,
flags (bit 1: a per-CPU buffer, whose events carry u32 vpid, u32 vtid after the
8-byte header)}; class rows {func_id u16, kind u8, 0, fixed_bytes u16, result_off i16,
cmd_off i16, 0 x6}; function rows {name_off u32, layer u16, 0}; host rows
{name_off u32, 0}; NUL-terminated strings; fixed-size packets at a 256-aligned
offset, each a 32-byte header {magic "PKT1", stream_id, ts_begin u64,
content_bytes, n_events, seq, discarded} then events.
"""
from __future__ import annotations

import struct
from dataclasses import dataclass, field

TRACE_MAGIC = 0x54504854
PACKET_MAGIC = 0x31544B50
EXT_BIT = 1 << 27
DELTA_LIMIT = 1 << 27

ENTRY, EXIT, DEV_BEGIN, DEV_END, SAMPLE = 0, 1, 2, 3, 4


@dataclass
class Ev:
    """One event with an absolute timestamp (stream_events input)."""
    cls: int
    ts: int
    payload: bytes = b""
    result: int | None = None
    cmd: int | None = None
    force_ext: bool = False
    ctx: tuple | None = None  # (vpid, vtid) of an event of a per-CPU buffer


@dataclass
class _Class:
    func: int
    kind: int
    fixed: int
    result_off: int
    cmd_off: int


@dataclass
class TraceBuilder:
    packet_bytes: int = 256
    hosts: list = field(default_factory=list)
    funcs: list = field(default_factory=list)
    classes: list = field(default_factory=list)
    streams: list = field(default_factory=list)
    packets: list = field(default_factory=list)  # raw packet byte strings in file order
    _seq: dict = field(default_factory=dict)

    def add_host(self, name: str) -> int:
        self.hosts.append(name)
        return len(self.hosts) - 1

    def add_func(self, name: str, layer: int = 0) -> int:
        self.funcs.append((name, layer))
        return len(self.funcs) - 1

    def add_class(self, func: int, kind: int, fixed: int = 0, result_off: int = -1, cmd_off: int = -1) -> int:
        self.classes.append(_Class(func, kind, fixed, result_off, cmd_off))
        return len(self.classes) - 1

    def add_call_func(self, name: str, layer: int = 0, entry_fixed: int = 0, exit_fixed: int = 4):
        """A function with an ENTRY class and an EXIT class (i32 result at offset 0)."""
        f = self.add_func(name, layer)
        e = self.add_class(f, ENTRY, entry_fixed)
        x = self.add_class(f, EXIT, exit_fixed, 0 if exit_fixed >= 4 else -1)
        return f, e, x

    def add_stream(self, host: int, pid: int, tid: int, flags: int = 0) -> int:
        self.streams.append((host, pid, tid, flags))
        return len(self.streams) - 1

    # ------------------------------------------------------------ events
    def encode_event(self, cls: int, delta: int = 0, ext_ts: int | None = None, payload: bytes = b"",
                     result: int | None = None, cmd: int | None = None, raw_tsw: int | None = None,
                     var_len: int | None = None, fixed_override: bytes | None = None,
                     ctx: tuple | None = None) -> bytes:
        """Encodes one event.  ``raw_tsw``/``var_len``/``fixed_override`` allow malformed encodings;
        ``ctx`` = (vpid, vtid) adds the per-CPU context after the 8-byte header."""
        c = self.classes[cls] if cls < len(self.classes) else _Class(0, ENTRY, 0, -1, -1)
        if raw_tsw is not None:
            tsw = raw_tsw
        elif ext_ts is not None:
            tsw = EXT_BIT
        else:
            assert 0 <= delta < DELTA_LIMIT
            tsw = delta
        vl = len(payload) if var_len is None else var_len
        out = struct.pack("<IHH", tsw, cls, vl)
        if ctx is not None:
            out += struct.pack("<II", ctx[0] & 0xFFFFFFFF, ctx[1] & 0xFFFFFFFF)
        if ext_ts is not None:
            out += struct.pack("<Q", ext_ts & 0xFFFFFFFFFFFFFFFF)
        if fixed_override is not None:
            fixed = bytearray(fixed_override)
        else:
            fixed = bytearray(b"\xab" * c.fixed)
            if c.result_off >= 0:
                fixed[c.result_off:c.result_off + 4] = struct.pack("<i", result or 0)
            if c.cmd_off >= 0:
                fixed[c.cmd_off:c.cmd_off + 8] = struct.pack("<Q", (cmd or 0) & 0xFFFFFFFFFFFFFFFF)
        out += bytes(fixed) + payload
        out += b"\x00" * ((-len(out)) % 4)
        return out

    def raw_packet(self, stream_id: int, ts_begin: int, event_bytes: list, seq: int | None = None,
                   discarded: int = 0, n_events: int | None = None, content_bytes: int | None = None,
                   magic: int = PACKET_MAGIC) -> None:
        content = b"".join(event_bytes)
        cb = len(content) if content_bytes is None else content_bytes
        ne = len(event_bytes) if n_events is None else n_events
        if seq is None:
            seq = self._seq.get(stream_id, 0)
        self._seq[stream_id] = seq + 1
        hdr = struct.pack("<IIQIIII", magic, stream_id, ts_begin & 0xFFFFFFFFFFFFFFFF, cb, ne, seq, discarded)
        pkt = hdr + content
        if len(pkt) > self.packet_bytes:
            pkt = pkt[: self.packet_bytes]
        pkt += b"\x00" * (self.packet_bytes - len(pkt))
        self.packets.append(pkt)

    def stream_events(self, stream_id: int, events: list, ts_begin: int | None = None,
                      discarded_at: dict | None = None) -> list:
        """Packs events (absolute ts) into packets; returns the raw packets (not yet placed).

        ``discarded_at`` maps a packet ordinal to its discarded counter.
        Call ``place`` to append them to the file (interleaving is up to the caller).
        """
        cap = self.packet_bytes - 32
        pkts = []
        cur = []
        used = 0
        prev = events[0].ts if (ts_begin is None and events) else (ts_begin or 0)
        begin = prev
        for ev in events:
            def enc(prev_ts):
                d = ev.ts - prev_ts
                if ev.force_ext or d < 0 or d >= DELTA_LIMIT:
                    return self.encode_event(ev.cls, ext_ts=ev.ts, payload=ev.payload, result=ev.result, cmd=ev.cmd,
                                             ctx=ev.ctx)
                return self.encode_event(ev.cls, delta=d, payload=ev.payload, result=ev.result, cmd=ev.cmd,
                                         ctx=ev.ctx)
            b = enc(prev)
            if used + len(b) > cap:
                pkts.append((begin, cur))
                cur, used, begin = [], 0, prev
                b = enc(prev)
            assert len(b) <= cap, "event larger than a packet"
            cur.append(b)
            used += len(b)
            prev = ev.ts
        if cur:
            pkts.append((begin, cur))
        out = []
        for i, (tb, evs) in enumerate(pkts):
            disc = (discarded_at or {}).get(i, 0)
            out.append((stream_id, tb, evs, disc))
        return out

    def place(self, packed: list) -> None:
        for (sid, tb, evs, disc) in packed:
            self.raw_packet(sid, tb, evs, discarded=disc)

    # -------------------------------------------------------------- file
    def build(self, header_patch: dict | None = None) -> bytes:
        """Serialises the trace.  ``header_patch`` maps a header byte offset to a
        (struct format, value) pair written over the finished header."""
        strings = bytearray()
        func_off, host_off = [], []
        for (name, _layer) in self.funcs:
            func_off.append(len(strings))
            strings += name.encode() + b"\x00"
        for name in self.hosts:
            host_off.append(len(strings))
            strings += name.encode() + b"\x00"
        off = 128
        st_off = off
        off += 16 * len(self.streams)
        cl_off = off
        off += 16 * len(self.classes)
        fn_off = off
        off += 8 * len(self.funcs)
        ho_off = off
        off += 8 * len(self.hosts)
        str_off = off
        off += len(strings)
        pk_off = (off + 255) & ~255
        hdr = bytearray(128)
        struct.pack_into("<IHHIIIII", hdr, 0, TRACE_MAGIC, 1, 128, self.packet_bytes, len(self.streams),
                         len(self.classes), len(self.funcs), len(self.hosts))
        struct.pack_into("<QQQQQQQQ", hdr, 32, len(self.packets), st_off, cl_off, fn_off, ho_off, str_off,
                         len(strings), pk_off)
        body = bytearray()
        for (h, pid, tid, flags) in self.streams:
            body += struct.pack("<IIII", h, pid, tid, flags)
        for c in self.classes:
            body += struct.pack("<HBBHhhHI", c.func, c.kind, 0, c.fixed, c.result_off, c.cmd_off, 0, 0)
        for i, (_name, layer) in enumerate(self.funcs):
            body += struct.pack("<IHH", func_off[i], layer, 0)
        for i in range(len(self.hosts)):
            body += struct.pack("<II", host_off[i], 0)
        body += strings
        out = bytes(hdr) + bytes(body)
        out += b"\x00" * (pk_off - len(out))
        out += b"".join(self.packets)
        if header_patch:
            ba = bytearray(out)
            for o, (fmt, v) in header_patch.items():
                struct.pack_into(fmt, ba, o, v)
            out = bytes(ba)
        return out


def pack_stream_arrays(tb: TraceBuilder, stream_id: int, ts, cls, result=None, ts_begin: int | None = None) -> int:
    """Vectorised packing of one stream's events (no payloads) into ``tb``.

    ts: u64 absolute timestamps (stream order); cls: class ids; result: i32
    written at each class's result offset (0 where None).  Appends the packets
    to ``tb`` in stream order and returns how many were written.
    """
    import numpy as np

    ts = np.asarray(ts, dtype=np.uint64)
    cls = np.asarray(cls, dtype=np.int64)
    n = len(ts)
    if n == 0:
        return 0
    res = np.zeros(n, dtype=np.int32) if result is None else np.asarray(result, dtype=np.int32)
    fixed = np.array([c.fixed for c in tb.classes], dtype=np.int64)
    roff = np.array([c.result_off for c in tb.classes], dtype=np.int64)
    tb0 = int(ts[0]) if ts_begin is None else int(ts_begin)
    prev = np.empty(n, dtype=np.uint64)
    prev[0] = tb0
    prev[1:] = ts[:-1]
    delta = ts - prev                      # wraps when negative
    ext = (ts < prev) | (delta >= np.uint64(DELTA_LIMIT))
    size = 8 + 8 * ext.astype(np.int64) + fixed[cls]
    cap = tb.packet_bytes - 32
    assert int(size.max()) <= cap
    csum = np.concatenate([[0], np.cumsum(size)])
    starts = [0]
    while starts[-1] < n:
        s = starts[-1]
        e = int(np.searchsorted(csum, csum[s] + cap, side="right")) - 1
        starts.append(max(e, s + 1))
    starts = np.array(starts, dtype=np.int64)
    n_pk = len(starts) - 1
    pk_of = np.repeat(np.arange(n_pk), np.diff(starts))
    off_in = csum[:-1] - csum[starts[:-1]][pk_of]
    P = tb.packet_bytes
    buf = np.zeros(n_pk * P, dtype=np.uint8)
    w32 = buf.view("<u4")
    pos = (pk_of * P + 32 + off_in) // 4
    tsw = np.where(ext, np.uint64(EXT_BIT), delta).astype(np.uint32)
    w32[pos] = tsw
    w32[pos + 1] = cls.astype(np.uint32)          # var_len = 0 in the high half
    epos = pos[ext] + 2
    w32[epos] = (ts[ext] & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    w32[epos + 1] = (ts[ext] >> np.uint64(32)).astype(np.uint32)
    has_r = roff[cls] >= 0
    rpos = pos + 2 + 2 * ext.astype(np.int64) + roff[cls] // 4
    w32[rpos[has_r]] = res[has_r].view(np.uint32)
    # packet headers
    first_ts_prev = prev[starts[:-1]]
    hdr = (np.arange(n_pk) * P) // 4
    w32[hdr] = PACKET_MAGIC
    w32[hdr + 1] = stream_id
    w32[hdr + 2] = (first_ts_prev & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    w32[hdr + 3] = (first_ts_prev >> np.uint64(32)).astype(np.uint32)
    w32[hdr + 4] = (csum[starts[1:]] - csum[starts[:-1]]).astype(np.uint32)
    w32[hdr + 5] = np.diff(starts).astype(np.uint32)
    seq0 = tb._seq.get(stream_id, 0)
    w32[hdr + 6] = (seq0 + np.arange(n_pk)).astype(np.uint32)
    tb._seq[stream_id] = seq0 + n_pk
    for k in range(n_pk):
        tb.packets.append(buf[k * P:(k + 1) * P].tobytes())
    return n_pk
