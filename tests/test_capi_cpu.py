"""The C-ABI library loads on a machine without a GPU and exports every
symbol include/mmref.h declares; host-side argument checks need no device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"MMREF_API\s+[\w\s\*]+?\b(mm_\w+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def mm():
    from paper_1308_4011_b300 import build
    build.build()
    from paper_1308_4011_b300 import mmref
    return mmref


def test_every_declared_symbol_is_exported(mm):
    declared = _declared()
    assert len(declared) >= 10
    lib = ctypes.CDLL(mm.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(mm.EXPORTED) == sorted(declared)


def test_abi_version_and_status_strings(mm):
    assert mm.abi_version() == 1
    assert mm._lib.mm_status_string(mm.MM_EINVAL) == b"invalid argument"
    assert mm._lib.mm_status_string(mm.MM_EBUDGET) == b"memory budget exceeded"


def test_host_side_argument_checks(mm):
    """Errors found before any device work: NULL desc, bad sizes, bad ptr kind."""
    h = ctypes.c_void_p()
    assert mm._lib.mm_load_system(None, None, ctypes.byref(h)) == mm.MM_EINVAL
    assert b"non-NULL" in mm._lib.mm_last_error()
    d = mm._Desc(0, 0, 0, 0, 0, 0, None, None, None, None, None, None, 1, 0)
    assert mm._lib.mm_load_system(ctypes.byref(d), None, ctypes.byref(h)) == mm.MM_EINVAL
    d = mm._Desc(3, 2, 0, 7, 0, 0, None, None, None, None, None, None, 1, 0)
    assert mm._lib.mm_load_system(ctypes.byref(d), None, ctypes.byref(h)) == mm.MM_EINVAL
    assert b"ptr_kind" in mm._lib.mm_last_error()
    assert mm._lib.mm_compute_metrics(None, None, None, 0) == mm.MM_EINVAL
    assert h.value is None


def test_dtypes_match_header_sizes(mm):
    assert mm.CLASS_METRICS_DTYPE.itemsize == 64
    assert mm.METHOD_METRICS_DTYPE.itemsize == 16
    assert mm.MOVE_EVAL_DTYPE.itemsize == 16
    assert mm.MOVE_DTYPE.itemsize == 24
