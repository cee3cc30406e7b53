"""thapi_decode (the decode step made visible) vs the oracle's decode, field
by field, and vs the generator's record of what it wrote."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import tracegen as tg
from tests import _malformed
from tracegen.handbuilt import ENTRY, EXIT, Ev, TraceBuilder

pytestmark = pytest.mark.gpu
FIELDS = ("ts", "cmd", "stream_id", "class_id", "var_len", "result", "ext", "kind", "func_id")


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2504_03683_b300 import thapi
    assert torch.cuda.is_available()
    c = thapi.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("name,over", [
    ("tiny", {}),
    ("large", dict(total_calls=60_000, n_hosts=1, pids_per_host=2, tids_per_pid=3, p_long_gap=0.01, p_ext=0.02,
                   p_sample=0.05, packet_bytes=1024, seed=5)),
    ("large", dict(total_calls=40_000, n_hosts=1, pids_per_host=2, tids_per_pid=2, packet_bytes=256, p_drop=0.01,
                   seed=6)),
    ("large", dict(total_calls=50_000, n_hosts=1, pids_per_host=2, tids_per_pid=2, packet_bytes=32768, seed=7)),
    ("device", dict(total_calls=30_000, n_hosts=1, pids_per_host=2, tids_per_pid=2, n_device_streams=3, seed=8)),
])
def test_decode_matches_oracle_and_generator(ctx, name, over):
    b, _calls, truth = tg.generate(tg.preset(name, **over), truth=True)
    got = ctx.decode(b)
    ref = oracle.decode(b)
    assert len(got) == len(ref) == len(truth)
    for f in FIELDS:
        assert np.array_equal(got[f], ref[f]), f
        assert np.array_equal(got[f], truth[f]), f


def test_decode_ext_boundary(ctx):
    tb = TraceBuilder(packet_bytes=256)
    h = tb.add_host("h")
    f, e, x = tb.add_call_func("f")
    s = tb.add_stream(h, 1, 1)
    t0 = 10**18
    evs = [Ev(e, t0), Ev(x, t0 + (1 << 27) - 1), Ev(e, t0 + (1 << 27) - 1 + (1 << 27)), Ev(x, t0 + 3 * (1 << 27) - 2)]
    tb.place(tb.stream_events(s, evs, ts_begin=t0))
    got = ctx.decode(tb.build())
    assert list(got["ts"]) == [ev.ts for ev in evs]
    assert list(got["ext"]) == [0, 0, 1, 0]
    assert list(got["kind"]) == [ENTRY, EXIT, ENTRY, EXIT]


@pytest.mark.parametrize("name,trace", _malformed.cases(), ids=[c[0] for c in _malformed.cases()])
def test_decode_errors_match_oracle(ctx, name, trace):
    from paper_2504_03683_b300 import thapi
    o = oracle.run(trace)
    if o.code == oracle.OK:
        got = ctx.decode(trace)
        ref = oracle.decode(trace)
        assert all(np.array_equal(got[f], ref[f]) for f in FIELDS)
        return
    with pytest.raises(thapi.ThapiError) as ei:
        ctx.decode(trace)
    assert ei.value.code == o.code, (name, ei.value.code, o.code)
    if o.loc[0] > 0:
        assert ei.value.location == o.loc, name
