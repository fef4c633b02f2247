"""The C-ABI library loads on a machine without a GPU and exports every entry
point declared in include/lrh.h (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "lrh.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lrh_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ["lrh_create", "lrh_destroy", "lrh_step", "lrh_bound", "lrh_get_messages", "lrh_set_messages",
              "lrh_evaluate", "lrh_restart", "lrh_set_options", "lrh_get_info", "lrh_get_pairs",
              "lrh_get_region_values", "lrh_synchronize", "lrh_strerror", "lrh_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2609_40336_b300 import build, _lib
    build.build()
    lib = ctypes.CDLL(_lib.LIB_PATH)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding declares exactly the header's entry points
    assert sorted(_lib.SIGNATURES) == declared_symbols()


def test_strerror_without_gpu():
    from paper_2609_40336_b300 import _lib
    lib = _lib.load()
    assert lib.lrh_strerror(-8) == b"unsupported region size"
    assert lib.lrh_strerror(0) == b"ok"


# ---------------------------------------------------------------- host-side validation
# These return before any device call, so they run on a machine without a GPU.
import numpy as np  # noqa: E402

import lrh_gen as g  # noqa: E402


def _create(p):
    from paper_2609_40336_b300 import Solver
    return Solver(p)


def _code(p):
    from paper_2609_40336_b300._lib import LrhError
    with pytest.raises(LrhError) as ei:
        _create(p)
    return ei.value.code


def test_region_beyond_eight_sites_is_rejected():
    p = g.Problem(9, [tuple(range(9))], [(0, 1)], [g.lattices.ZZ[None]])
    assert _code(p) == -1


def test_duplicate_region_is_rejected():
    p = g.Problem(2, [(0, 1), (0, 1)], [(0, 1)], [g.lattices.ZZ[None]])
    assert _code(p) == -3


def test_unsorted_region_is_rejected():
    p = g.Problem(2, [(1, 0)], [(0, 1)], [g.lattices.ZZ[None]])
    assert _code(p) == -1


def test_term_outside_every_region_is_rejected():
    p = g.Problem(3, [(0, 1), (1, 2)], [(0, 2)], [g.lattices.ZZ[None]])
    assert _code(p) == -3


def test_non_hermitian_term_is_rejected():
    m = np.zeros((1, 4, 4), np.complex128)
    m[0, 0, 1] = 1.0
    p = g.Problem(2, [(0, 1)], [(0, 1)], [m])
    assert _code(p) == -2


def test_bad_options_are_rejected():
    from paper_2609_40336_b300 import Solver
    from paper_2609_40336_b300._lib import LrhError
    p = g.Problem(2, [(0, 1)], [(0, 1)], [g.lattices.ZZ[None]])
    with pytest.raises(LrhError) as ei:
        Solver(p, variant="nesterov", beta=-1.0)
    assert ei.value.code == -1
