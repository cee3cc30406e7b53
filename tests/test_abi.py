"""The C ABI library loads and exports every entry point its header declares
(no compute calls: runs without a GPU)."""
import os
import re

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
    for code in range(9):
        assert thapi.thapi_strerror(code)
    assert thapi.thapi_strerror(99) == "unknown status"


def test_struct_sizes_match_header():
    import ctypes
    assert thapi.ROW_DTYPE.itemsize == 56
    assert thapi.INTERVAL_DTYPE.itemsize == 24
    assert ctypes.sizeof(thapi.Diag) == 64
    assert ctypes.sizeof(thapi.DeviceDiag) == 64
    assert ctypes.sizeof(thapi.TraceInfo) == 8 * 6 + 4 * 6 + 16 + 16
    assert ctypes.sizeof(thapi.LoadTiming) == 4 * 8 + 8 * 4 + 4 * 4 + 8 * 2
