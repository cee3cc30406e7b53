"""The C ABI library loads and exports every entry point its header declares
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2504_03683_b300 import thapi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(thapi_[a-z_0-9]+)\s*\(", src))
    return names


def test_header_declares_the_binding_surface():
    declared = _declared()
    assert declared == set(thapi.EXPORTED), declared ^ set(thapi.EXPORTED)


def test_library_exports_every_declared_symbol():
    lib = thapi.library()
    for name in _declared():
        assert hasattr(lib, name), name


def test_strerror_is_static_and_total():
    for code in range(10):
        assert thapi.thapi_strerror(code) != "unknown status"
    assert thapi.thapi_strerror(99) == "unknown status"


def test_struct_sizes_match_header():
    import ctypes
    assert thapi.ROW_DTYPE.itemsize == 56
    assert thapi.INTERVAL_DTYPE.itemsize == 24
    assert ctypes.sizeof(thapi.Diag) == 64
    assert ctypes.sizeof(thapi.DeviceDiag) == 64
    assert ctypes.sizeof(thapi.TraceInfo) == 8 * 6 + 4 * 6 + 16 + 16
    assert ctypes.sizeof(thapi.LoadTiming) == 4 * 8 + 8 * 4 + 4 * 4 + 8 * 2 + 4 * 2 + 4 * 2


def test_struct_layouts_match_the_header(tmp_path):
    """Every ABI struct's size and field offsets, compiled from include/thapi.h
    with the host C compiler, equal the binding's ctypes / numpy layouts."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_2504_03683_b300 import thapi
    layouts = {
        "thapi_tally_row": thapi.ROW_DTYPE, "thapi_interval": thapi.INTERVAL_DTYPE,
        "thapi_event": thapi.EVENT_DTYPE, "thapi_diag": thapi.Diag, "thapi_device_diag": thapi.DeviceDiag,
        "thapi_trace_info": thapi.TraceInfo, "thapi_load_timing": thapi.LoadTiming,
        "thapi_request": thapi.Request, "thapi_result": thapi.Result, "thapi_server_stats": thapi.ServerStats,
    }
    want = {}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "thapi.h"', "int main(void) {"]
    for st, lay in layouts.items():
        if isinstance(lay, np.dtype):
            fields = [(f, lay.fields[f][1]) for f in lay.names]
            size = lay.itemsize
        else:
            fields = [(f, getattr(lay, f).offset) for f, _t in lay._fields_]
            size = ctypes.sizeof(lay)
        want[st] = [size] + [o for _f, o in fields]
        args = ", ".join(["sizeof(%s)" % st] + ["offsetof(%s, %s)" % (st, f) for f, _o in fields])
        lines.append('  printf("' + st + " %zu" * (len(fields) + 1) + '\\n", ' + args + ");")
    lines += ["  return 0;", "}"]
    (tmp_path / "layout.c").write_text("\n".join(lines))
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-I" + inc, str(tmp_path / "layout.c"), "-o", str(tmp_path / "layout")], check=True)
    out = subprocess.run([str(tmp_path / "layout")], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, out):
        name, *vals = line.split()
        assert [int(v) for v in vals] == want[name], name
