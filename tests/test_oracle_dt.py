"""Time step (Eq. 55 with the Courant and diffusion limits of the reading in the
oracle's header) against closed forms built here from the box geometry and the
parameters: a uniform state has sound speed c_s everywhere, so each level's limit is
min_d CFL dx_d / (c_s + |V_d|) and CFL_diff / (2 chi sum_d dx_d^-2), and the coarse
step is min_l (level limit) 2^l.  A hot cell (four times the internal energy, twice
the sound speed) on the finest level lowers that level's limit by the known amount.
CPU only."""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_1812_03191_gb300 import inputs as I

N, NL = 24, 3
LO, HI = (-6.0, -4.0, -8.0), (6.0, 4.0, 8.0)   # unequal cell sizes per axis
FLOW = (0.6, 0.0, -0.8)


def _cell_sizes(level):
    return [(HI[d] - LO[d]) / N / 2**level for d in range(3)]


def _limits(p, cs_cell):
    """per-level (advective, diffusive) limits of a uniform state with the given sound
    speed; None where the limit does not apply"""
    V = [p["mach"] * p["cs"] * f for f in FLOW]
    out = []
    for l in range(NL):
        dx = _cell_sizes(l)
        adv = min(p["cfl"] * dx[d] / (cs_cell + abs(V[d])) for d in range(3)) \
            if p["hydro_on"] else None
        dif = p["cfl_diff"] / (2 * p["chi"] * sum(1 / h**2 for h in dx)) \
            if p["chi"] > 0 else None
        out.append((adv, dif))
    return out


def _level_dt(lim):
    return min(x for x in lim if x is not None)


@pytest.mark.parametrize("chi", [0.0, 0.05, 5.0])
def test_uniform_state_time_step(chi):
    """chi = 0: sound crossing only; 5: the diffusion limit everywhere; 0.05: the
    advective limit on coarse levels, diffusion on the finest (it scales as dx^2)"""
    p = I.base_params(GM=0.0, L=0.0, chi=chi, mach=1.3, flow_dir=FLOW)
    o = Oracle(NL, N, LO, HI, I.DEFAULT_G, p)
    dt, per_level = o.compute_dt()
    want = [_level_dt(lim) for lim in _limits(p, p["cs"])]
    assert np.allclose(per_level, want, rtol=1e-14, atol=0), (per_level, want)
    assert dt == pytest.approx(min(w * 2**l for l, w in enumerate(want)), rel=1e-14)
    if chi == 0.05:  # both limits take part, as intended
        kinds = [int(lim[1] < lim[0]) for lim in _limits(p, p["cs"])]
        assert kinds[0] == 0 and kinds[-1] == 1, kinds


def test_hot_cell_sets_its_level_limit():
    p = I.base_params(GM=0.0, L=0.0, chi=0.0, mach=0.7, flow_dir=FLOW)
    o = Oracle(NL, N, LO, HI, I.DEFAULT_G, p)
    e = o.get_field(NL - 1, 1)
    e[5, 7, 11] *= 4.0
    o.set_field(NL - 1, 1, e)
    _, per_level = o.compute_dt()
    cold = _limits(p, p["cs"])
    hot = _limits(p, 2.0 * p["cs"])
    assert per_level[0] == pytest.approx(cold[0][0], rel=1e-14)
    assert per_level[-1] == pytest.approx(hot[-1][0], rel=1e-14)
    assert per_level[-1] < cold[-1][0]


def test_fixed_step_overrides_the_limits():
    p = I.base_params(GM=0.0, L=0.0, chi=1.0, dt_fixed=1.25e-3)
    o = Oracle(NL, N, LO, HI, I.DEFAULT_G, p)
    assert o.compute_dt()[0] == 1.25e-3
    o.step(1)
    assert o.last_dt == 1.25e-3 and math.isclose(o.t, 1.25e-3)
