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
