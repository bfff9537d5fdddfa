"""The C-ABI library loads and exports every symbol include/dfnest.h declares; the
host-side validation rejects bad input before any device work.  CPU only."""
import ctypes as C
import os
import re

import pytest

from paper_1812_03191_gb300 import binding
from paper_1812_03191_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return binding.load()


def test_header_and_binding_agree():
    hdr = open(os.path.join(ROOT, "include", "dfnest.h")).read()
    declared = set(re.findall(r"\b(df_[a-z0-9_]+)\s*\(", hdr))
    assert declared == set(binding.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in binding.EXPORTS:
        assert hasattr(lib, name), name


def test_invalid_geometry_rejected_without_gpu(lib):
    h = C.c_void_p()
    n = (C.c_int * 3)(30, 32, 32)  # not a multiple of 4
    lo = (C.c_double * 3)(-1, -1, -1)
    hi = (C.c_double * 3)(1, 1, 1)
    assert lib.df_create(C.byref(h), 1, n, lo, hi, 8, 0, 0, None) == binding.DF_EINVAL
    assert b"n[0]" in lib.df_last_error()
    n2 = (C.c_int * 3)(32, 32, 32)
    assert lib.df_create(C.byref(h), 0, n2, lo, hi, 8, 0, 0, None) == binding.DF_EINVAL
    assert lib.df_create(C.byref(h), 1, n2, hi, lo, 8, 0, 0, None) == binding.DF_EINVAL
    assert lib.df_create(C.byref(h), 1, n2, lo, hi, 8, 7, 0, None) == binding.DF_EINVAL
    big = (C.c_int * 3)(1024, 1024, 1024)
    assert lib.df_create(C.byref(h), 1, big, lo, hi, 8, 0, 0, None) == binding.DF_EINVAL
    assert lib.df_step(None, 1, None) == binding.DF_EINVAL
    t = C.c_double()
    assert lib.df_step(None, 1, C.byref(t)) == binding.DF_EINVAL


def test_problem_statement_calls_validate_without_gpu(lib):
    """df_create_levels / df_step / df_pool_force (the hot path's contract calls)
    reject bad input on the host, before any device work."""
    h = C.c_void_p()
    lo = (C.c_double * 3)(-8, -8, -8)
    hi = (C.c_double * 3)(8, 8, 8)
    alloc = binding._ALLOC_FN(lambda nbytes, user: None)
    # one callback without the other
    assert lib.df_create_levels(C.byref(h), 3, 64, lo, hi, 0, 0, None,
                                C.cast(alloc, C.c_void_p), None, None) == binding.DF_EINVAL
    assert b"together" in lib.df_last_error()
    # N not a multiple of 4; no levels; too many levels; unknown precision
    assert lib.df_create_levels(C.byref(h), 3, 30, lo, hi, 0, 0, None, None, None,
                                None) == binding.DF_EINVAL
    assert lib.df_create_levels(C.byref(h), 0, 64, lo, hi, 0, 0, None, None, None,
                                None) == binding.DF_EINVAL
    assert lib.df_create_levels(C.byref(h), 17, 64, lo, hi, 0, 0, None, None, None,
                                None) == binding.DF_EINVAL
    assert lib.df_create_levels(C.byref(h), 3, 64, lo, hi, 5, 0, None, None, None,
                                None) == binding.DF_EINVAL
    assert not h.value
    F = (C.c_double * 3)()
    t = C.c_double()
    assert lib.df_pool_force(None, 0, F, C.byref(t)) == binding.DF_EINVAL


def test_xi_search_matches_appendix_example(lib):
    # Appendix A: flat wins iff K > 2/3 (two equal-cost levels)
    assert binding.xi_search([1.0, 0.6], [1, 1])[1] == [2]
    assert binding.xi_search([1.0, 0.7], [1, 1])[1] == [1]
    assert binding.xi_search([1.0, 0.9, 0.4], [1, 1, 1])[1] == [1, 2]
