"""The paper's worked tally (Sec. 4.3) reproduced by the oracle at the printed precision."""
import oracle
from tests import _paper_trace as pt


def test_paper_hiplz_table_reproduced():
    trace, golden, names = pt.build()
    r = oracle.run(trace, want_intervals=False)
    assert r.code == oracle.OK
    assert r.diag["unmatched_entries"] == r.diag["unmatched_exits"] == r.diag["mismatched_pairs"] == 0
    got = pt.render(r.rows, names)
    for g in golden:
        assert got[g["name"]] == (g["time"], g["pct"], str(g["calls"]), g["avg"], g["min"], g["max"]), g["name"]
    # the printed order is Time descending
    shown = [g["name"] for g in golden]
    by_time = sorted(shown, key=lambda n: -int(r.rows[[names[int(f)] == n for f in r.rows["func_id"]]][0]["total_ns"]))
    assert by_time == shown


def _parse_table(text):
    """{name: (Time, Time%, Calls, Average, Min, Max)} from a rendered table."""
    out = {}
    for line in text.splitlines()[2:]:
        cells = [c.strip() for c in line.strip(" |").split("|")]
        if len(cells) == 7:
            out[cells[0]] = tuple(cells[1:])
    return out


def test_product_renderer_reproduces_paper_table_from_rows():
    """The package's table renderer, fed the oracle's rows, prints the paper's values
    in the paper's order (Time descending)."""
    from paper_2504_03683_b300.render import tally_table
    trace, golden, names = pt.build()
    r = oracle.run(trace, want_intervals=False)
    text = tally_table(r.rows, names)
    got = _parse_table(text)
    for g in golden:
        assert got[g["name"]] == (g["time"], g["pct"], str(g["calls"]), g["avg"], g["min"], g["max"]), g["name"]
    order = [ln.split("|")[0].strip() for ln in text.splitlines()[2:]]
    assert order[:len(golden)] == [g["name"] for g in golden]


def test_event_lines_render_decoded_events():
    """The pretty-printer turns decoded events into one line each: timestamp,
    hostname, vpid / vtid, function_kind and the fields every class has."""
    from paper_2504_03683_b300.render import event_lines
    from tests._device_trace import build
    from tests._util import stream_table
    b, ids = build()
    ev = oracle.decode(b)
    st = stream_table(b)
    names = ["launchKernel", "memcpyAsync", "deviceWork"]
    lines = event_lines(ev, names, ["n0"], st)
    assert len(lines) == len(ev)
    assert lines[0].startswith("1000000 n0 vpid: 7, vtid: 7 - launchKernel_entry: { cmd: 0x000000000000000a")
    assert lines[1] == "1000010 n0 vpid: 7, vtid: 7 - launchKernel_exit: { result: 0, payload_bytes: 0 }"
    dev = [ln for ln in lines if "deviceWork_device_begin" in ln]
    assert dev[0].startswith("1000100 n0 vpid: 900, vtid: 1 - deviceWork_device_begin: { cmd: 0x000000000000000a")


def test_self_table_and_layer_summary_on_the_layered_case():
    """The hip-over-Level-Zero case by hand (self times 25, 22 + 45, 8 ns): the
    layer summary splits the 100 ns of the outer call between the HIP layer (25)
    and the Level Zero layer (75)."""
    import oracle
    from paper_2504_03683_b300.render import layer_summary, self_table
    from tracegen.handbuilt import Ev, TraceBuilder
    tb = TraceBuilder(packet_bytes=256)
    h = tb.add_host("h")
    hip, eh, xh = tb.add_call_func("hipDeviceSynchronize", layer=0)
    ze, ez, xz = tb.add_call_func("zeEventHostSynchronize", layer=1)
    lf, el, xl = tb.add_call_func("zeLeaf", layer=1)
    s = tb.add_stream(h, 1, 1)
    evs = [Ev(eh, 1000), Ev(ez, 1010), Ev(el, 1012), Ev(xl, 1020, result=0), Ev(xz, 1040, result=0),
           Ev(ez, 1050), Ev(xz, 1095, result=0), Ev(xh, 1100, result=2)]
    tb.place(tb.stream_events(s, evs, ts_begin=1000))
    r = oracle.run(tb.build())
    names = ["hipDeviceSynchronize", "zeEventHostSynchronize", "zeLeaf"]
    layers = [0, 1, 1]
    text = self_table(r.rows, r.self_rows, names, layers)
    lines = text.splitlines()
    assert lines[2].split("|")[0].strip() == "zeEventHostSynchronize"  # largest self time first
    hip_line = [ln for ln in lines if ln.strip().startswith("hipDeviceSynchronize")][0]
    cells = [c.strip() for c in hip_line.split("|")]
    assert cells[1:7] == ["0", "100ns", "25ns", "25.00%", "1", "25ns"]
    txt, per = layer_summary(r.self_rows, layers, layer_names=["HIP", "ZE"])
    assert per == {0: (25, 1), 1: (75, 3)}
    assert txt.splitlines()[2].split("|")[0].strip() == "ZE"
