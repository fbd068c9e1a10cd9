"""The C-ABI library loads and exports every function include/*.h declares
(no GPU needed: symbols only, no compute calls)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names += re.findall(r"^\s*(?:int|void|const char\*)\s+(smmo_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libsmmo():
    from paper_1908_05845_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_calls():
    names = declared()
    for n in ("smmo_heap_create", "smmo_class_register", "smmo_bulk_new", "smmo_parallel_do",
              "smmo_enumerate_live", "smmo_compact"):
        assert n in names


def test_every_declared_symbol_exported(libsmmo):
    missing = [n for n in declared() if not hasattr(libsmmo, n)]
    assert not missing, missing


def test_status_strings(libsmmo):
    libsmmo.smmo_status_string.restype = ctypes.c_char_p
    assert libsmmo.smmo_status_string(0) == b"ok"
    assert b"double free" in libsmmo.smmo_status_string(-7)


def test_method_table(libsmmo):
    mid = ctypes.c_int()
    assert libsmmo.smmo_method_lookup(b"test.add_i32", ctypes.byref(mid)) == 0
    assert libsmmo.smmo_method_lookup(b"no.such.method", ctypes.byref(mid)) == -1


def test_create_rejects_bad_args(libsmmo):
    h = ctypes.c_void_p()
    assert libsmmo.smmo_heap_create(None, None, ctypes.c_size_t(1 << 20), None, ctypes.byref(h)) == -1
    # misaligned buffer pointer is rejected before any CUDA call
    assert libsmmo.smmo_heap_create(None, ctypes.c_void_p(0x1001), ctypes.c_size_t(1 << 20), None,
                                    ctypes.byref(h)) == -1
