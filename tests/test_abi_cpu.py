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
    declared = set(re.findall(r"\b(df_[a-z_]+)\s*\(", hdr))
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
    assert lib.df_step(None, 1) == binding.DF_EINVAL


def test_xi_search_matches_appendix_example(lib):
    # Appendix A: flat wins iff K > 2/3 (two equal-cost levels)
    assert binding.xi_search([1.0, 0.6], [1, 1])[1] == [2]
    assert binding.xi_search([1.0, 0.7], [1, 1])[1] == [1]
    assert binding.xi_search([1.0, 0.9, 0.4], [1, 1, 1])[1] == [1, 2]
