"""Malformed traces, one per validation rule, plus precedence cases."""
from __future__ import annotations

import struct

from tracegen.handbuilt import TraceBuilder


def _base():
    tb = TraceBuilder(packet_bytes=256)
    h = tb.add_host("h")
    _f, e, x = tb.add_call_func("f")
    s0 = tb.add_stream(h, 1, 1)
    s1 = tb.add_stream(h, 1, 2)
    return tb, e, x, s0, s1


def _good_packets(tb, e, x, s0):
    tb.raw_packet(s0, 0, [tb.encode_event(e, 1), tb.encode_event(x, 2)])


def cases():
    out = []

    tb, e, x, s0, s1 = _base()
    _good_packets(tb, e, x, s0)
    good = tb.build()
    out.append(("good", good))
    out.append(("file_truncated_header", good[:100]))
    out.append(("file_bad_magic", b"XXXX" + good[4:]))
    out.append(("file_bad_version", tb.build({4: ("<H", 2)})))
    out.append(("file_packet_size", tb.build({8: ("<I", 300)})))
    out.append(("file_packets_beyond_end", tb.build({32: ("<Q", 5)})))
    out.append(("file_packets_misaligned", tb.build({88: ("<Q", 300)})))
    out.append(("file_truncated_tail", good[:-10]))

    for name, mut in [("class_kind", lambda tb, e, x: setattr(tb.classes[e], "kind", 9)),
                      ("class_fixed", lambda tb, e, x: setattr(tb.classes[x], "fixed", 6)),
                      ("class_result_off", lambda tb, e, x: setattr(tb.classes[x], "result_off", 4)),
                      ("class_cmd_off", lambda tb, e, x: setattr(tb.classes[x], "cmd_off", 0))]:
        tb, e, x, s0, s1 = _base()
        mut(tb, e, x)
        _good_packets(tb, e, x, s0)
        out.append((name, tb.build()))
    tb, e, x, s0, s1 = _base()
    tb.streams[s1] = (7, 1, 2, 0)
    out.append(("stream_host", tb.build()))

    tb, e, x, s0, s1 = _base()
    tb.raw_packet(s0, 0, [tb.encode_event(e, 1, raw_tsw=0x10000000)])
    tb.raw_packet(s1, 0, [tb.encode_event(e, 1)], magic=0xDEAD)
    out.append(("header_before_content", tb.build()))

    good_ev = None
    for case in ("tsw_high_bits", "bad_class", "ext_with_delta", "event_overruns", "header_overruns",
                 "count_mismatch", "count_more"):
        tb, e, x, s0, s1 = _base()
        _good_packets(tb, e, x, s0)
        good_ev = tb.encode_event(e, 3)
        if case == "tsw_high_bits":
            tb.raw_packet(s1, 0, [good_ev, tb.encode_event(x, raw_tsw=0x20000005)])
        elif case == "bad_class":
            tb.raw_packet(s1, 0, [good_ev, struct.pack("<IHH", 1, 77, 0)])
        elif case == "ext_with_delta":
            tb.raw_packet(s1, 0, [good_ev, tb.encode_event(x, raw_tsw=(1 << 27) | 4, ext_ts=50)])
        elif case == "event_overruns":
            tb.raw_packet(s1, 0, [good_ev, tb.encode_event(x, 1, payload=b"\x00" * 8)],
                          content_bytes=len(good_ev) + 12)
        elif case == "header_overruns":
            tb.raw_packet(s1, 0, [good_ev, b"\x01\x00\x00\x00"], n_events=1)
        elif case == "count_mismatch":
            tb.raw_packet(s1, 0, [good_ev, tb.encode_event(x, 1)], n_events=1)
        elif case == "count_more":
            tb.raw_packet(s1, 0, [good_ev, tb.encode_event(x, 1)], n_events=3)
        out.append((case, tb.build()))

    tb, e, x, s0, s1 = _base()
    tb.raw_packet(s0, 0, [tb.encode_event(e, 1)], seq=5)
    tb.raw_packet(s0, 0, [tb.encode_event(x, 1)], seq=5)
    out.append(("seq_not_increasing", tb.build()))
    tb, e, x, s0, s1 = _base()
    tb.raw_packet(9, 0, [tb.encode_event(e, 1)])
    out.append(("stream_out_of_range", tb.build()))
    tb, e, x, s0, s1 = _base()
    tb.raw_packet(s0, 0, [tb.encode_event(e, 1)], content_bytes=6)
    out.append(("content_unaligned", tb.build()))
    tb, e, x, s0, s1 = _base()
    tb.raw_packet(s0, 0, [tb.encode_event(e, 1)], content_bytes=240)
    out.append(("content_too_big", tb.build()))
    # a later packet's content error must not beat an earlier one
    tb, e, x, s0, s1 = _base()
    tb.raw_packet(s0, 0, [tb.encode_event(e, 1), tb.encode_event(x, raw_tsw=0x30000000)])
    tb.raw_packet(s1, 0, [struct.pack("<IHH", 1, 99, 0)])
    out.append(("first_content_error_wins", tb.build()))
    # speculative walk lands mid-event: a payload that looks like headers
    tb, e, x, s0, s1 = _base()
    fake = struct.pack("<IHH", 0, e, 0) * 6
    tb.raw_packet(s0, 0, [tb.encode_event(e, 1, payload=fake), tb.encode_event(x, 2), b"\x05\x00\x00\x00"],
                  n_events=2)
    out.append(("garbage_tail_after_fake_headers", tb.build()))
    return out
