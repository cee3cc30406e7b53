"""Two THPT traces with the same class, function and host tables joined into
one trace (input construction only): the second trace's streams follow the
first's (its packets' stream ids shifted), and its packets follow the first's
packets.  Streams of the two halves may share (host, pid, tid), so a tally of
the joined trace combines their rows — which is what a merge of the two
halves' tallies must give.
"""
from __future__ import annotations

import struct

import numpy as np


def _hdr(b: bytes):
    (magic, ver, hb, P, n_streams, n_classes, n_funcs, n_hosts, _z) = struct.unpack_from("<IHHIIIIII", b, 0)
    (n_packets, st_off, cl_off, fn_off, ho_off, str_off, str_bytes, pk_off) = struct.unpack_from("<8Q", b, 32)
    return dict(P=P, n_streams=n_streams, n_classes=n_classes, n_funcs=n_funcs, n_hosts=n_hosts,
                n_packets=n_packets, st_off=st_off, cl_off=cl_off, fn_off=fn_off, ho_off=ho_off,
                str_off=str_off, str_bytes=str_bytes, pk_off=pk_off)


def concat(a, b) -> np.ndarray:
    a = bytes(a)
    b = bytes(b)
    ha, hb = _hdr(a), _hdr(b)
    assert ha["P"] == hb["P"]
    for k in ("n_classes", "n_funcs", "n_hosts"):
        assert ha[k] == hb[k], k
    assert a[ha["cl_off"]:ha["cl_off"] + 16 * ha["n_classes"]] == b[hb["cl_off"]:hb["cl_off"] + 16 * hb["n_classes"]]
    P = ha["P"]
    S = ha["n_streams"] + hb["n_streams"]
    streams = a[ha["st_off"]:ha["st_off"] + 16 * ha["n_streams"]] + b[hb["st_off"]:hb["st_off"] + 16 * hb["n_streams"]]
    classes = a[ha["cl_off"]:ha["cl_off"] + 16 * ha["n_classes"]]
    funcs = a[ha["fn_off"]:ha["fn_off"] + 8 * ha["n_funcs"]]
    hosts = a[ha["ho_off"]:ha["ho_off"] + 8 * ha["n_hosts"]]
    strings = a[ha["str_off"]:ha["str_off"] + ha["str_bytes"]]
    off = 128
    st_off = off
    off += len(streams)
    cl_off = off
    off += len(classes)
    fn_off = off
    off += len(funcs)
    ho_off = off
    off += len(hosts)
    str_off = off
    off += len(strings)
    pk_off = (off + 255) & ~255
    n_packets = ha["n_packets"] + hb["n_packets"]
    head = bytearray(pk_off)
    struct.pack_into("<IHHIIIIII", head, 0, 0x54504854, 1, 128, P, S, ha["n_classes"], ha["n_funcs"], ha["n_hosts"], 0)
    struct.pack_into("<8Q", head, 32, n_packets, st_off, cl_off, fn_off, ho_off, str_off, len(strings), pk_off)
    head[st_off:st_off + len(streams)] = streams
    head[cl_off:cl_off + len(classes)] = classes
    head[fn_off:fn_off + len(funcs)] = funcs
    head[ho_off:ho_off + len(hosts)] = hosts
    head[str_off:str_off + len(strings)] = strings
    pa = np.frombuffer(a, dtype=np.uint8, count=ha["n_packets"] * P, offset=ha["pk_off"])
    pb = np.frombuffer(b, dtype=np.uint8, count=hb["n_packets"] * P, offset=hb["pk_off"]).copy()
    pbv = pb.reshape(hb["n_packets"], P)
    sid = pbv[:, 4:8].copy().view("<u4").reshape(-1) + np.uint32(ha["n_streams"])
    pbv[:, 4:8] = sid.view(np.uint8).reshape(-1, 4)
    return np.concatenate([np.frombuffer(bytes(head), dtype=np.uint8), pa, pb])


def concat_batch(traces) -> np.ndarray:
    """N traces with the same packet size, class table and function names
    joined into one trace the way a batch load combines them: trace i's
    streams follow the earlier traces' (its packets' stream ids shifted), its
    hosts likewise (host ids shifted, its host names appended to the string
    table), its packets after the earlier traces' packets; the class and
    function tables are trace 0's."""
    bs = [bytes(t) for t in traces]
    hs = [_hdr(b) for b in bs]
    P = hs[0]["P"]
    a, ha = bs[0], hs[0]
    classes = a[ha["cl_off"]:ha["cl_off"] + 16 * ha["n_classes"]]
    funcs = a[ha["fn_off"]:ha["fn_off"] + 8 * ha["n_funcs"]]
    strings = bytearray(a[ha["str_off"]:ha["str_off"] + ha["str_bytes"]])
    streams, hosts, packets = bytearray(), bytearray(), []
    s_base = h_base = 0
    for i, (b, h) in enumerate(zip(bs, hs)):
        assert h["P"] == P and b[h["cl_off"]:h["cl_off"] + 16 * h["n_classes"]] == classes
        str_base = 0
        if i > 0:
            str_base = len(strings)
            strings += b[h["str_off"]:h["str_off"] + h["str_bytes"]]
        for k in range(h["n_hosts"]):
            off, z = struct.unpack_from("<II", b, h["ho_off"] + 8 * k)
            hosts += struct.pack("<II", off + str_base, z)
        for k in range(h["n_streams"]):
            host, pid, tid, flags = struct.unpack_from("<IIII", b, h["st_off"] + 16 * k)
            streams += struct.pack("<IIII", host + h_base, pid, tid, flags)
        pk = np.frombuffer(b, dtype=np.uint8, count=h["n_packets"] * P, offset=h["pk_off"]).copy()
        v = pk.reshape(h["n_packets"], P)
        sid = v[:, 4:8].copy().view("<u4").reshape(-1) + np.uint32(s_base)
        v[:, 4:8] = sid.view(np.uint8).reshape(-1, 4)
        packets.append(pk)
        s_base += h["n_streams"]
        h_base += h["n_hosts"]
    n_packets = sum(h["n_packets"] for h in hs)
    off = 128
    st_off = off
    off += len(streams)
    cl_off = off
    off += len(classes)
    fn_off = off
    off += len(funcs)
    ho_off = off
    off += len(hosts)
    str_off = off
    off += len(strings)
    pk_off = (off + 255) & ~255
    head = bytearray(pk_off)
    struct.pack_into("<IHHIIIIII", head, 0, 0x54504854, 1, 128, P, s_base, ha["n_classes"], ha["n_funcs"], h_base, 0)
    struct.pack_into("<8Q", head, 32, n_packets, st_off, cl_off, fn_off, ho_off, str_off, len(strings), pk_off)
    head[st_off:st_off + len(streams)] = streams
    head[cl_off:cl_off + len(classes)] = classes
    head[fn_off:fn_off + len(funcs)] = funcs
    head[ho_off:ho_off + len(hosts)] = hosts
    head[str_off:str_off + len(strings)] = strings
    return np.concatenate([np.frombuffer(bytes(head), dtype=np.uint8)] + packets)
