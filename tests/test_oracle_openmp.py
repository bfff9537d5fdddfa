"""The OpenMP build of the oracle (the same C file compiled with -fopenmp, used to
time the oracle on all host cores) computes the same bits as the plain build: its
parallel loops write disjoint elements, and every sum stays serial.  CPU only."""
import numpy as np
import pytest

import oracle
from oracle import Oracle
from paper_1812_03191_gb300 import inputs as I


@pytest.fixture(scope="module", autouse=True)
def _omp():
    try:
        oracle.build_oracle(omp=True)
    except Exception as exc:  # a compiler without OpenMP
        pytest.skip(f"no OpenMP build: {exc}")
    prev = oracle.threads()
    assert oracle.threads(3) == 3
    yield
    oracle.threads(prev)


def _perturb(runs, seed, amp=1e-2):
    """the same smooth perturbation on every level of every run"""
    for l in range(runs[0].n_levels):
        for f in range(5):
            base = runs[0].get_field(l, f)
            pert = I.smooth_perturbation(base.shape, seed + 17 * l + f, amp)
            val = base * (1 + pert) if f < 2 else base + pert
            for r in runs:
                r.set_field(l, f, val)
    for l in range(runs[0].n_levels - 1):
        for r in runs:
            r.commup(l)


def _same(a, b, steps):
    a.step(steps)
    b.step(steps)
    assert a.t == b.t
    for l in range(a.n_levels):
        for f in range(5):
            assert np.array_equal(a.get_full(l, f), b.get_full(l, f)), (l, f)
    assert np.array_equal(a.force(), b.force())


def test_nested_run_is_bitwise_the_plain_build():
    """three nested levels with diffusion, luminosity, the Eq. 55-56 search and a
    perturbed state: every padded element and the force agree bit for bit"""
    p = I.base_params(GM=0.02, eps=0.3, chi=0.5, L=0.03, lum_sigma=0.3, mach=0.9,
                      xi_mode=1)
    args = (3, 24, (-6.0,) * 3, (6.0,) * 3, I.DEFAULT_G, p)
    a, b = Oracle(*args), Oracle(*args, omp=True)
    _perturb([a, b], seed=5)
    _same(a, b, 3)


def test_quadrant_ground_and_viscosity_are_bitwise_the_plain_build():
    """mirror planes, a ground level of its own size and SubStep2 viscosity"""
    cfg = I.quadrant(n=24, n_levels=3, half=6.0, mach=1.5, quarter=True, GM=0.05, chi=0.3,
                     L=0.02, av_c2=2.0)
    args = (cfg["n_levels"], cfg["n"], cfg["lo"], cfg["hi"], cfg["G"], cfg["params"])
    a = Oracle(*args, n0=cfg["n0"])
    b = Oracle(*args, n0=cfg["n0"], omp=True)
    _perturb([a, b], seed=9)
    _same(a, b, 3)
