"""The C ABI: the library builds, loads and exports every function that
include/*.h declares; host-side behaviour that needs no GPU."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        for m in re.finditer(r"\b(sj_[a-z0-9_]+)\s*\(", text):
            if not re.search(r"typedef[^;]*\(\*\s*" + m.group(1) + r"\s*\)", text):
                names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1908_11740_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("sj_create", "sj_destroy", "sj_partition", "sj_join", "sj_count", "sj_join_into",
                 "sj_free", "sj_part_free", "sj_strerror", "sj_last_error"):
        assert need in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_1908_11740_gb300 import sj

    bound = {s[0] for s in sj.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_strerror(lib):
    lib.sj_strerror.restype = ctypes.c_char_p
    assert lib.sj_strerror(0) == b"ok"
    assert b"invalid" in lib.sj_strerror(1)
    assert lib.sj_strerror(999) == b"unknown status"


def test_create_rejects_bad_device(lib):
    h = ctypes.c_void_p()
    # device -1 never exists; without a GPU every device is rejected
    assert lib.sj_create(ctypes.byref(h), -1, None) == 1
    assert h.value is None
    assert lib.sj_create(None, 0, None) == 1


def test_null_context_is_rejected(lib):
    lib.sj_join.restype = ctypes.c_int
    assert lib.sj_join(None, None, 0, None, 0, None, None, None, None) == 1
    assert lib.sj_count(None, None, 0, None, 0, None, None) == 1
    assert lib.sj_destroy(None) == 1


def test_null_context_is_rejected_by_every_join_entry(lib):
    P, I64, F = ctypes.c_void_p, ctypes.c_int64, ctypes.c_float
    lib.sj_distance_join.argtypes = [P, P, I64, P, I64, F, P, P, P, P, P]
    lib.sj_distance_join_into.argtypes = [P, P, I64, P, I64, F, P, P, P, I64, P, P]
    lib.sj_join_host_many.argtypes = [P, ctypes.c_int, P, P, P, P, P, P, P, P, P]
    assert lib.sj_distance_join(None, None, 0, None, 0, 0.1, None, None, None, None, None) == 1
    assert lib.sj_distance_join_into(None, None, 0, None, 0, 0.1, None, None, None, 0, None, None) == 1
    assert lib.sj_join_host_many(None, 0, None, None, None, None, None, None, None, None, None) == 1
