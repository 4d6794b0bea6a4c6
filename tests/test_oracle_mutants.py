"""The oracle's pins must catch plausible mistakes in it.

Each case copies the oracle's C source to a temporary directory, plants one
mistake (a dropped term, a wrong comparison, a wrong index, a transposed
output ...), builds it, and checks that at least one pin fails against the
mutant.  The pins used are the ones of test_oracle_pins: the hand-built
Fig. 1 instance, the lattice closed form, and routes that do not share the
mutated code.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1908_11740_gb300 import inputs
from test_oracle_pins import _count_1d, _lattice, load_fig1

SRC = os.path.join(os.path.dirname(oracle.__file__), "sj_oracle.c")

# (name, original text, mutated text); each original must occur exactly once.
MUTANTS = [
    ("scan bound open (r pivot)", "R[i].xu >= S[k].xl", "R[i].xu > S[k].xl"),
    ("scan bound open (s pivot)", "S[j].xu >= R[k].xl", "S[j].xu > R[k].xl"),
    ("scan skips current s", "for (int64_t k = j; k < ns", "for (int64_t k = j + 1; k < ns"),
    ("y test open", "return ryl <= syu && syl <= ryu;", "return ryl < syu && syl <= ryu;"),
    ("y test drops a term", "return ryl <= syu && syl <= ryu;", "return ryl <= syu;"),
    ("Eq. 1 strict", ">= d->col &&", "> d->col &&"),
    ("Eq. 1 min instead of max", "float my = r->yl > s->yl ? r->yl : s->yl;",
     "float my = r->yl < s->yl ? r->yl : s->yl;"),
    ("no duplicate test", "if (!d->on) return 1;", "return 1;"),
    ("replication drops last column", "for (int cx = cx0; cx <= cx1; cx++) {",
     "for (int cx = cx0; cx < cx1 + (cx0 == cx1); cx++) {"),
    ("wrong tile row index", "d.row = (int)(t / nx);", "d.row = (int)(t % ny);"),
    ("transposed output (s pivot)", "res_push(res, R[k].id, S[j].id);", "res_push(res, S[j].id, R[k].id);"),
    ("sort by upper endpoint", "if (x->xl < y->xl) return -1;\n    if (x->xl > y->xl) return 1;",
     "if (x->xu < y->xu) return -1;\n    if (x->xu > y->xu) return 1;"),
]


def _build_mutant(tmp_path, orig, new):
    src = open(SRC).read()
    assert src.count(orig) == 1, orig
    path = tmp_path / "m.c"
    path.write_text(src.replace(orig, new))
    so = tmp_path / "libm.so"
    subprocess.check_call(["gcc", *oracle.CFLAGS, "-o", str(so), str(path), "-lm"])
    return ctypes.CDLL(str(so))


def _run(lib, fn, R, S, *grid):
    P, I64, I, F = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_float
    lib.orc_res_count.restype = I64
    lib.orc_res_count.argtypes = [P]
    lib.orc_res_copy.argtypes = [P, P]
    lib.orc_res_free.argtypes = [P]
    R = np.ascontiguousarray(R, np.float32)
    S = np.ascontiguousarray(S, np.float32)
    if fn == "pbsm":
        lib.orc_pbsm_ex.restype = P
        lib.orc_pbsm_ex.argtypes = [P, I64, P, I64, I, I, F, F, F, F, P, P, P, P]
        res = lib.orc_pbsm_ex(R.ctypes.data, len(R), S.ctypes.data, len(S), *grid, None, None, None, None)
    else:
        lib.orc_sweep.restype = P
        lib.orc_sweep.argtypes = [P, I64, P, I64, P]
        res = lib.orc_sweep(R.ctypes.data, len(R), S.ctypes.data, len(S), None)
    n = lib.orc_res_count(res)
    out = np.empty((n, 2), np.int32)
    if n:
        lib.orc_res_copy(res, out.ctypes.data)
    lib.orc_res_free(res)
    return out


def _pins_hold(lib):
    """True when the mutant passes every pin (i.e. the mutation is missed)."""
    R, S, pairs, meta = load_fig1()
    for fn, grid in (("pbsm", (3, 3, 0.0, 0.0, 1.0, 1.0)), ("sweep", ())):
        if not np.array_equal(_run(lib, fn, R, S, *grid), pairs[:, :2]):
            return False
    n, u, d = 40, 1.0 / 256, 4
    for a_u, b_u, dx_u, dy_u in [(8, 4, 0, 0), (5, 7, 3, -2), (4, 4, 4, 0)]:
        LR = _lattice(n, d * u, a_u * u, 0.25, 0.25)
        LS = _lattice(n, d * u, b_u * u, 0.25 + dx_u * u, 0.25 + dy_u * u)
        want = _count_1d(n, -((dx_u + b_u) // d), (a_u - dx_u) // d) * \
            _count_1d(n, -((dy_u + b_u) // d), (a_u - dy_u) // d)
        for fn, grid in (("pbsm", (16, 16, 0.0, 0.0, 1.0, 1.0)), ("sweep", ())):
            if len(_run(lib, fn, LR, LS, *grid)) != want:
                return False
    R, S = inputs.degenerate_pair(300, 250, seed=4)
    want = oracle.brute(R, S)          # the unmutated definition
    for fn, grid in (("pbsm", (7, 7, 0.0, 0.0, 1.0, 1.0)), ("sweep", ())):
        if not np.array_equal(_run(lib, fn, R, S, *grid), want):
            return False
    return True


@pytest.mark.parametrize("name,orig,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, name, orig, new):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    lib = _build_mutant(tmp_path, orig, new)
    assert not _pins_hold(lib), f"pins missed the planted mistake: {name}"


def test_unmutated_oracle_passes_pins(tmp_path):
    lib = _build_mutant(tmp_path, "static int y_intersects", "static int y_intersects")
    assert _pins_hold(lib)
