"""The paper's worked tally (Sec. 4.3) through the CUDA path and the package's
table renderer, names from the trace's string table."""
import pytest

from tests import _paper_trace as pt
from tests.test_paper_table import _parse_table

pytestmark = pytest.mark.gpu


def test_gpu_tally_renders_paper_table():
    from paper_2504_03683_b300 import thapi
    from paper_2504_03683_b300.render import tally_table, trace_names
    trace, golden, _names = pt.build()
    with thapi.Context(0) as ctx:
        tid = ctx.load(trace)
        rows, diag = ctx.tally(tid)
        funcs, hosts = trace_names(ctx, tid)
        ctx.free(tid)
    assert diag["unmatched_entries"] == diag["unmatched_exits"] == diag["mismatched_pairs"] == 0
    got = _parse_table(tally_table(rows, funcs))
    for g in golden:
        assert got[g["name"]] == (g["time"], g["pct"], str(g["calls"]), g["avg"], g["min"], g["max"]), g["name"]


def test_gpu_self_table_with_layers_from_the_trace():
    """Self rows and function layers through the ABI, rendered: the layer
    summary of the GPU rows equals the one of the oracle's rows."""
    import oracle
    from paper_2504_03683_b300 import thapi
    from paper_2504_03683_b300.render import func_layers, layer_summary, self_table, trace_names
    from tracegen.handbuilt import Ev, TraceBuilder
    tb = TraceBuilder(packet_bytes=256)
    h = tb.add_host("h")
    hip, eh, xh = tb.add_call_func("hipDeviceSynchronize", layer=0)
    ze, ez, xz = tb.add_call_func("zeEventHostSynchronize", layer=1)
    lf, el, xl = tb.add_call_func("zeLeaf", layer=1)
    s = tb.add_stream(h, 1, 1)
    evs = []
    t = 1000
    for k in range(50):
        evs += [Ev(eh, t), Ev(ez, t + 10), Ev(el, t + 12), Ev(xl, t + 20 + k % 3, result=0),
                Ev(xz, t + 40, result=0), Ev(ez, t + 50), Ev(xz, t + 95, result=k % 4 == 0), Ev(xh, t + 100, result=0)]
        t += 200
    tb.place(tb.stream_events(s, evs, ts_begin=1000))
    trace = tb.build()
    with thapi.Context(0) as ctx:
        ctx.set_self_time(True)
        tid = ctx.load(trace)
        rows, _d = ctx.tally(tid)
        srows = ctx.self_tally(tid)
        funcs, _hosts = trace_names(ctx, tid)
        layers = func_layers(ctx, tid)
        ctx.free(tid)
    assert layers == [0, 1, 1]
    r = oracle.run(trace)
    assert self_table(rows, srows, funcs, layers) == self_table(r.rows, r.self_rows, funcs, layers)
    _t, per = layer_summary(srows, layers)
    assert per == layer_summary(r.self_rows, layers)[1]
    assert per[0][0] + per[1][0] == int(r.rows[r.rows["func_id"] == hip]["total_ns"][0])
