"""Index arithmetic of the kernels, checked on the CPU by brute force: the CommUp
tiling, the box decode's multiply-shift division and the CommFlux record layout
(host-callable helpers in internal.h, compiled as host code with nvcc; no GPU
needed)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1812_03191_gb300", "csrc")


def _run_check(tmp_path, name):
    """compile tests/<name>.cu as a host program and run it: it prints OK or FAIL"""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / name)
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    "-o", exe, os.path.join(ROOT, "tests", name + ".cu")],
                   check=True, capture_output=True, timeout=300)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout[-2000:]
    assert out.stdout.startswith("OK ")


def test_commup_tiles_cover_the_ghost_hosts_exactly(tmp_path):
    _run_check(tmp_path, "commup_tiles_check")


def test_box_decode_division_is_exact(tmp_path):
    """Box::magic: (t m) >> s == t / d for t < 2^31 at every quotient boundary tried
    and at pseudo-random t, divisors 1..4096 and sampled plane sizes up to 1.5 Mi"""
    _run_check(tmp_path, "magic_div_check")


def test_commflux_record_layout_is_one_to_one(tmp_path):
    """rec_index maps (axis, side, quantity, sub-cycle, transverse position) one to one
    onto [0, rec_elems) for cubic and uneven padded shapes"""
    _run_check(tmp_path, "rec_index_check")
