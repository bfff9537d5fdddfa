"""Host-side pieces of the heating-force ladder (no GPU)."""
import math

import pytest

from paper_1812_03191_gb300 import ladder


def test_plume_length_time_and_increment():
    # Eq. 7, Eq. 9, Eq. 24 at the Sec. 4.1 set-up (gamma 1.4, chi 0.1, Mach 3)
    assert ladder.lam(0.1, 1.4, 3.0) == pytest.approx(0.1 / 4.2)
    assert ladder.tau(0.1, 1.4, 3.0) == pytest.approx(ladder.lam(0.1, 1.4, 3.0) ** 2 / 0.1)
    assert ladder.eq24_increment(1.4, 1e-3, 2e-4, 0.1, 3.0) == pytest.approx(
        0.4 * 1e-3 * 2e-4 * math.log(2) / 0.9)


def test_fixed_step_respects_every_level():
    hot, cold, half = ladder.setup()
    assert half == pytest.approx(100 * ladder.lam(0.1, 1.4, 3.0))
    assert hot["L"] == 2e-4 and cold["L"] == 0.0 and hot["eps"] == 0.0
    for nl in (4, 5, 6, 7):
        dt = ladder.fixed_dt(nl, 32, half, hot)
        for l in range(nl):
            dx = 2 * half / 32 / 2**l
            lvl = dt / 2**l  # level l advances by the coarse step / 2^l
            assert lvl <= 0.44 * dx / 4.0 + 1e-15
            assert lvl <= 0.44 * dx * dx / 0.6 + 1e-15
        # diffusion on the finest level binds: each added level quarters the finest
        # step and the coarse step halves
        if nl > 4:
            assert dt == pytest.approx(ladder.fixed_dt(nl - 1, 32, half, hot) / 2)
