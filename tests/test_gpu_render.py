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
