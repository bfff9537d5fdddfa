"""A ground level with its own cell count (Sec. 4.1.1: a ground level of twice the
cells per axis of the nested levels, so that the first nested level covers a quarter
of the ground's extent).  Pins of the oracle's hierarchy against geometry built here
from first principles: the cell halves per level, level 1 spans [lo, hi] / 4 and
level l >= 2 spans [lo, hi] 2^-(l+1).  CPU only."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1812_03191_gb300 import inputs as I

RHO, ENE, VX, VY, VZ = range(5)
G = I.DEFAULT_G
HALF = 6.0
N = 24          # nested levels
N0 = 2 * N      # ground


def level_box(level):
    """half-width and cell size of a level of the quarter hierarchy"""
    if level == 0:
        return HALF, 2 * HALF / N0
    h = HALF / 2 ** (level + 1)
    return h, 2 * h / N


def positions(level, field, padded):
    h, dx = level_box(level)
    n = N0 if level == 0 else N
    idx = np.arange(n + 2 * G) - G if padded else np.arange(n)
    cen = -h + (idx + 0.5) * dx
    face = -h + idx * dx
    axes = [cen, cen, cen]
    if field >= VX:
        axes[field - VX] = face
    z, y, x = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return x, y, z


def make(nl, **over):
    return Oracle(nl, N, (-HALF,) * 3, (HALF,) * 3, G, I.base_params(**over), n0=N0)


def covered(level, nl):
    """mask of the active cells of a level that its child covers, from coordinates"""
    x, y, z = positions(level, RHO, False)
    if level == nl - 1:
        return np.zeros(x.shape, dtype=bool)
    hc, _ = level_box(level + 1)
    return (np.abs(x) < hc) & (np.abs(y) < hc) & (np.abs(z) < hc)


def composite(o, nl, field):
    tot = 0.0
    for l in range(nl):
        _, dx = level_box(l)
        a = o.get_field(l, field)
        tot += a[~covered(l, nl)].sum() * dx**3
    return tot


def test_level_one_covers_the_middle_quarter():
    """the covered ground cells are the middle quarter of each axis, and each
    nested level covers the middle half of its parent"""
    nl = 3
    m0 = covered(0, nl)
    assert m0.sum() == (N0 // 4) ** 3
    idx = np.argwhere(m0)
    assert idx.min() == 3 * N0 // 8 and idx.max() == 3 * N0 // 8 + N0 // 4 - 1
    assert covered(1, nl).sum() == (N // 2) ** 3


def test_commup_reproduces_linear_fields_with_a_ground_level():
    """CommUp from a ground of 2n cells into a level of n cells over a quarter of its
    extent: linear fields are reproduced exactly at the fine elements' positions"""
    o = make(2)
    coef = np.array([0.3, -0.7, 0.45, 1.1])
    for f in range(5):
        x, y, z = positions(0, f, True)
        o.set_full(0, f, coef[0] + 0.1 * f + coef[1] * x + coef[2] * y + coef[3] * z)
        o.set_full(1, f, np.full(o.full_shape(1), np.nan))
    o.commup(0)
    for f in range(5):
        x, y, z = positions(1, f, True)
        got = o.get_full(1, f)
        want = coef[0] + 0.1 * f + coef[1] * x + coef[2] * y + coef[3] * z
        filled = ~np.isnan(got)
        assert filled.sum() > 0.5 * got.size
        assert np.abs(got[filled] - want[filled]).max() < 1e-13, f


def test_uniform_flow_stays_uniform_with_a_ground_level():
    o = make(3, GM=0.0, L=0.0, chi=1.0, mach=0.7, flow_dir=(-0.6, 0.0, 0.8))
    init = [[o.get_field(l, f).copy() for f in range(5)] for l in range(3)]
    o.step(6)
    for l in range(3):
        for f in range(5):
            assert np.array_equal(o.get_field(l, f), init[l][f]), (l, f)


def _perturb(o, nl, seed, amp=1e-2):
    for l in range(nl):
        n = N0 if l == 0 else N
        for f in range(5):
            base = o.get_field(l, f)
            pert = I.smooth_perturbation((n, n, n), seed + 17 * l + f, amp)
            o.set_field(l, f, base * (1 + pert) if f < 2 else base + pert)
    for l in range(nl - 1):
        o.commup(l)


def test_mass_conserved_with_a_ground_level():
    """conservative transport and CommFlux keep the composite mass across the
    ground/first-level frontier too"""
    nl = 3
    o = make(nl, GM=0.0, L=0.0, chi=0.3, mach=0.8, flow_dir=(0.6, 0.8, 0.0),
             bc=(I.BC_PERIODIC,) * 6)
    _perturb(o, nl, seed=8)
    m0 = composite(o, nl, RHO)
    o.step(4)
    m1 = composite(o, nl, RHO)
    assert abs(m1 - m0) <= 1e-13 * abs(m0)
    assert o.t > 0


def test_energy_conserved_by_nested_diffusion_with_a_ground_level():
    nl = 3
    o = make(nl, GM=0.0, L=0.0, chi=0.8, hydro_on=0, bc=(I.BC_PERIODIC,) * 6)
    for l in range(nl):
        x, y, z = positions(l, RHO, False)
        e = o.get_field(l, ENE)
        o.set_field(l, ENE, e * (1 + 0.3 * np.exp(-(x**2 + y**2 + z**2) / (2 * 0.6**2))))
    for l in range(nl - 1):
        o.commup(l)
    e0 = composite(o, nl, ENE)
    o.step(4)
    e1 = composite(o, nl, ENE)
    assert abs(e1 - e0) <= 1e-13 * abs(e0)


def test_force_with_a_ground_level_matches_a_brute_force_sum():
    nl, GM, eps = 3, 0.013, 0.1
    o = make(nl, GM=GM, eps=eps)
    rng = np.random.default_rng(4)
    Fb = np.zeros(3, dtype=np.longdouble)
    for l in range(nl):
        n = N0 if l == 0 else N
        r = 1.0 + 0.05 * rng.standard_normal((n, n, n))
        o.set_field(l, RHO, r)
        x, y, z = (a.astype(np.longdouble) for a in positions(l, RHO, False))
        _, dx = level_box(l)
        r2 = x * x + y * y + z * z + np.longdouble(eps) ** 2
        w = np.longdouble(GM) * (r.astype(np.longdouble) - 1) * np.longdouble(dx) ** 3 / (
            r2 * np.sqrt(r2))
        w[covered(l, nl)] = 0
        Fb += np.array([(w * x).sum(), (w * y).sum(), (w * z).sum()])
    F = o.force()
    assert np.abs(F - Fb.astype(np.float64)).max() <= 1e-12 * np.abs(F).max()


def test_quadrant_with_a_ground_level_reproduces_the_whole_domain():
    """the paper's low-Mach geometry (Sec. 4.1.1): mirror planes through the
    perturber and a first level over a quarter of the ground, against the unfolded
    whole domain with the same ground"""
    p = I.base_params(gamma=1.4, mach=0.3, flow_dir=(0.0, 0.0, 1.0), GM=0.05, eps=0.0,
                      chi=0.3, L=0.02, lum_sigma=0.0,
                      bc=(I.BC_REFLECT,) * 4 + (I.BC_INFLOW,) * 2)
    full = Oracle(3, N, (-HALF,) * 3, (HALF,) * 3, G, p, n0=N0)
    part = Oracle(3, (N // 2, N // 2, N), (0.0, 0.0, -HALF), (HALF,) * 3, G, p,
                  n0=(N0 // 2, N0 // 2, N0))
    for _ in range(2):
        full.step(4)
        part.step(4)
    for l in range(3):
        n = N0 if l == 0 else N
        for f in range(5):
            a = full.get_field(l, f)[:, n // 2:, n // 2:]
            b = part.get_field(l, f)
            assert np.abs(a - b).max() <= 1e-12 * (2.0 if f == ENE else 1.0), (l, f)
    assert part.force()[2] == pytest.approx(full.force()[2], rel=1e-11)
    assert abs(part.force()[2]) > 1e-5
