"""Sod's shock tube (Sod 1978) against the exact solution of the Riemann problem: a
non-linear pin of the whole hydrodynamic scheme (kick, SubStep3, transport) and of
the SubStep2 artificial viscosity.  The exact solution is Toro's exact Riemann
solver (Toro 2009, ch. 4): Newton iteration on the star pressure, then sampling of
the wave pattern.  Oracle only (CPU)."""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_1812_03191_gb300 import inputs as I

G_AD = 1.4


def _pressure_function(p, rk, pk, ck, g):
    """Toro's f_K(p) and its derivative: shock branch for p > p_K, rarefaction else"""
    if p > pk:
        A, B = 2.0 / ((g + 1) * rk), (g - 1) / (g + 1) * pk
        return (p - pk) * math.sqrt(A / (p + B)), math.sqrt(A / (B + p)) * (1 - (p - pk) / (2 * (B + p)))
    r = p / pk
    return 2 * ck / (g - 1) * (r ** ((g - 1) / (2 * g)) - 1), r ** (-(g + 1) / (2 * g)) / (rk * ck)


def exact_riemann(x, t, left, right, x0, g=G_AD):
    """(rho, u, p) of the exact solution at positions x, time t"""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    p = 0.5 * (pl + pr)
    for _ in range(100):
        fl, dl = _pressure_function(p, rl, pl, cl, g)
        fr, dr = _pressure_function(p, rr, pr, cr, g)
        dp = (fl + fr + ur - ul) / (dl + dr)
        p = max(p - dp, 1e-14)
        if abs(dp) < 1e-15 * p:
            break
    u = 0.5 * (ul + ur) + 0.5 * (_pressure_function(p, rr, pr, cr, g)[0]
                                 - _pressure_function(p, rl, pl, cl, g)[0])
    out = np.empty((len(x), 3))
    for i, xi in enumerate(x):
        s = (xi - x0) / t
        if s < u:
            if p > pl:  # left shock
                sl = ul - cl * math.sqrt((g + 1) / (2 * g) * p / pl + (g - 1) / (2 * g))
                rs = rl * (p / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pl + 1)
                out[i] = (rs, u, p) if s > sl else (rl, ul, pl)
            else:  # left rarefaction
                head, tail = ul - cl, u - cl * (p / pl) ** ((g - 1) / (2 * g))
                if s < head:
                    out[i] = (rl, ul, pl)
                elif s > tail:
                    out[i] = (rl * (p / pl) ** (1 / g), u, p)
                else:
                    c = 2 / (g + 1) * (cl + (g - 1) / 2 * (ul - s))
                    out[i] = (rl * (c / cl) ** (2 / (g - 1)), 2 / (g + 1) * (cl + (g - 1) / 2 * ul + s),
                              pl * (c / cl) ** (2 * g / (g - 1)))
        else:
            if p > pr:  # right shock
                sr = ur + cr * math.sqrt((g + 1) / (2 * g) * p / pr + (g - 1) / (2 * g))
                rs = rr * (p / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pr + 1)
                out[i] = (rs, u, p) if s < sr else (rr, ur, pr)
            else:  # right rarefaction (not reached by Sod's data)
                head, tail = ur + cr, u + cr * (p / pr) ** ((g - 1) / (2 * g))
                if s > head:
                    out[i] = (rr, ur, pr)
                elif s < tail:
                    out[i] = (rr * (p / pr) ** (1 / g), u, p)
                else:
                    c = 2 / (g + 1) * (cr - (g - 1) / 2 * (ur - s))
                    out[i] = (rr * (c / cr) ** (2 / (g - 1)), 2 / (g + 1) * (-cr + (g - 1) / 2 * ur + s),
                              pr * (c / cr) ** (2 * g / (g - 1)))
    return out, p, u


def test_exact_solver_reproduces_sods_star_state():
    """The solver itself: Sod's data give p* = 0.30313, u* = 0.92745 (Toro, Table 4.3)."""
    _, p, u = exact_riemann(np.array([0.5]), 0.2, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.5)
    assert p == pytest.approx(0.30313, abs=2e-5) and u == pytest.approx(0.92745, abs=2e-5)


def sod_setup(av, nx=200, ny=8, steps=250):
    """x in [0, 1] with the diaphragm at 0.5, ny x ny periodic cells across; dt fixed
    at t = 0.2 / steps (Courant number ~0.35 on the fastest wave)."""
    p = I.base_params(gamma=G_AD, rho0=1.0, cs=1.2, mach=0.0, GM=0.0, eps=0.0, chi=0.0,
                      L=0.0, dt_fixed=0.2 / steps, av_c2=av,
                      bc=(I.BC_OUTFLOW, I.BC_OUTFLOW) + (I.BC_PERIODIC,) * 4)
    shape = (nx, ny, ny)
    lo, hi = (0.0, 0.0, 0.0), (1.0, ny / nx, ny / nx)
    xc = (np.arange(nx) + 0.5) / nx
    fields = [np.broadcast_to(np.where(xc < 0.5, 1.0, 0.125), (ny, ny, nx)).copy(),
              np.broadcast_to(np.where(xc < 0.5, 1.0, 0.1) / (G_AD - 1), (ny, ny, nx)).copy()]
    fields += [np.zeros((ny, ny, nx))] * 3
    return p, shape, lo, hi, fields, xc


def run_sod(av, steps=250):
    p, shape, lo, hi, fields, xc = sod_setup(av, steps=steps)
    o = Oracle(1, shape, lo, hi, I.DEFAULT_G, p)
    for f in range(5):
        o.set_field(0, f, fields[f])
    o.step(steps)
    return o, xc


def sod_errors(get, t, xc):
    """L1 errors of rho, p (cell centres) and u (lower x-faces) along the tube"""
    nx = len(xc)
    rho, e, vx = get(0)[0, 0], get(1)[0, 0], get(2)[0, 0]
    ex, _, _ = exact_riemann(xc, t, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.5)
    exf, _, _ = exact_riemann(xc - 0.5 / nx, t, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.5)
    return (np.abs(rho - ex[:, 0]).mean(), np.abs((G_AD - 1) * e - ex[:, 2]).mean(),
            np.abs(vx - exf[:, 1]).mean())


def test_sod_shock_tube_matches_the_exact_solution():
    """200 cells, t = 0.2: with the artificial viscosity (C2 = 2) the L1 errors of
    density, pressure and velocity are 0.0035, 0.0028 and 0.0068; without it the
    velocity error doubles (post-shock oscillations) -- the viscosity does its job."""
    o, xc = run_sod(2.0)
    er, ep, eu = sod_errors(lambda f: o.get_field(0, f), o.t, xc)
    assert o.t == pytest.approx(0.2, rel=1e-12)
    assert er < 0.005 and ep < 0.004 and eu < 0.009, (er, ep, eu)
    o0, _ = run_sod(0.0)
    er0, ep0, eu0 = sod_errors(lambda f: o0.get_field(0, f), o0.t, xc)
    assert er0 < 0.008 and eu0 > 1.4 * eu, (er0, eu0, eu)
    # the transverse directions stay exactly uniform and at rest
    for f in (3, 4):
        assert np.abs(o.get_field(0, f)).max() == 0.0
