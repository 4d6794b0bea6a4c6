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


def test_debug_build_exports_the_same_symbols():
    """The debug build with bounds checks (-DSJ_CHECK=1) compiles and loads
    with the same boundary."""
    from paper_1908_11740_gb300 import build

    dbg = ctypes.CDLL(build.build(check=True))
    missing = [n for n in declared_functions() if not hasattr(dbg, n)]
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


def test_plain_c_program_compiles_links_and_runs(lib, tmp_path):
    """include/sj.h is a C header: a C11 program includes it, links the
    library and calls it (calls that need no GPU)."""
    import shutil
    import subprocess

    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_1908_11740_gb300 import build

    so = build.build()
    src = tmp_path / "use_sj.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "sj.h"
int main(void) {
    sj_ctx *ctx = NULL;
    sj_grid g = {16, 16, 0.0f, 0.0f, 1.0f, 1.0f};
    sj_opts o = {SJ_TWO_PASS, 1, 0.25f, 0};
    sj_point p = {0.5f, 0.5f};
    int64_t n = 0;
    if (strcmp(sj_strerror(SJ_OK), "ok") != 0) return 1;
    if (sj_create(&ctx, -1, NULL) != SJ_EINVAL || ctx != NULL) return 2;
    if (sj_join(NULL, NULL, 0, NULL, 0, &g, &o, NULL, &n) != SJ_EINVAL) return 3;
    if (sj_distance_join(NULL, &p, 1, &p, 1, 0.1f, &g, &o, NULL, &n, NULL) != SJ_EINVAL) return 4;
    if (sizeof(sj_rect) != 16 || sizeof(sj_pair) != 8 || sizeof(sj_point) != 8) return 5;
    printf("ok\n");
    return 0;
}
''')
    exe = tmp_path / "use_sj"
    inc = os.path.join(ROOT, "include")
    libdir = os.path.dirname(so)
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-I", inc, str(src), "-o", str(exe),
                           "-L", libdir, "-l:" + os.path.basename(so), "-Wl,-rpath," + libdir])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0 and out.stdout.strip() == "ok", (out.returncode, out.stdout, out.stderr)
