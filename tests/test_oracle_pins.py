"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against an invariant, a closed form, a brute force or a
worked example -- never against the oracle itself.  CPU only.
"""
import math
import os

import numpy as np
import pytest

from oracle import Oracle, xi_search
from paper_1812_03191_gb300 import inputs as I

RHO, ENE, VX, VY, VZ = range(5)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def make(nl, n, half, G=I.DEFAULT_G, **over):
    if isinstance(half, (int, float)):
        lo, hi = (-half,) * 3, (half,) * 3
    else:
        lo, hi = tuple(-h for h in half), tuple(half)
    return Oracle(nl, n, lo, hi, G, I.base_params(**over))


def centres(o, level, n, lo, hi):
    """cell-centre coordinates of the active cells, shaped (nz, ny, nx)"""
    n = (n,) * 3 if isinstance(n, int) else n
    ax = []
    for d in range(3):
        dx = (hi[d] - lo[d]) / 2 ** level / n[d]
        ax.append(lo[d] / 2 ** level + (np.arange(n[d]) + 0.5) * dx)
    z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return x, y, z


# ---------------------------------------------------------------- T1

@pytest.mark.parametrize("rho0,av", [(1.0, 0.0), (1.3, 0.0), (1.0, 1.5)])
def test_uniform_flow_stays_uniform(rho0, av):
    """No perturber: a uniform wind is a steady solution of Eqs. 1-3 (and of the
    artificial viscosity, which needs compression)."""
    o = make(3, 24, 6.0, GM=0.0, L=0.0, chi=1.0, rho0=rho0, mach=0.7,
             flow_dir=(-0.6, 0.0, 0.8), av_c2=av)
    init = [[o.get_field(l, f).copy() for f in range(5)] for l in range(3)]
    o.step(8)
    for l in range(3):
        for f in range(5):
            a, b = o.get_field(l, f), init[l][f]
            if rho0 == 1.0:
                assert np.array_equal(a, b), (l, f)
            else:
                ulp = np.spacing(np.abs(b).max())
                assert np.abs(a - b).max() <= 4 * ulp, (l, f)


# ---------------------------------------------------------------- T2

def _perturb(o, nl, n, seed, amp=1e-2):
    for l in range(nl):
        for f in range(5):
            base = o.get_field(l, f)
            pert = I.smooth_perturbation((n, n, n), seed + 17 * l + f, amp)
            o.set_field(l, f, base * (1 + pert) if f < 2 else base + pert)
    for l in range(nl - 1):
        o.commup(l)


def _composite_sum(o, nl, n, field, vol0):
    tot = 0.0
    for l in range(nl):
        a = o.get_field(l, field)
        if l < nl - 1:
            m = np.ones_like(a, dtype=bool)
            q = n // 4
            m[q:q + n // 2, q:q + n // 2, q:q + n // 2] = False
            a = a[m]
        tot += a.sum() * vol0 / 8 ** l
    return tot


@pytest.mark.parametrize("nl", [1, 3])
def test_mass_conserved_periodic(nl):
    """Conservative transport with CommFlux keeps the composite mass (Sec. 3.2.3)."""
    n = 24
    o = make(nl, n, 6.0, GM=0.0, L=0.0, chi=0.3, mach=0.8, flow_dir=(0.6, 0.8, 0.0),
             bc=(I.BC_PERIODIC,) * 6)
    _perturb(o, nl, n, seed=5)
    vol0 = (12.0 / n) ** 3
    m0 = _composite_sum(o, nl, n, RHO, vol0)
    o.step(6)
    m1 = _composite_sum(o, nl, n, RHO, vol0)
    assert abs(m1 - m0) <= 1e-13 * abs(m0)
    # and the flow did move: the state is not trivially frozen
    assert o.t > 0


def test_energy_conserved_nested_diffusion():
    """Pure diffusion with CommFlux keeps the composite internal energy."""
    n, nl = 24, 3
    o = make(nl, n, 6.0, GM=0.0, L=0.0, chi=0.8, hydro_on=0, bc=(I.BC_PERIODIC,) * 6)
    for l in range(nl):
        x, y, z = centres(o, l, n, (-6,) * 3, (6,) * 3)
        e = o.get_field(l, ENE)
        o.set_field(l, ENE, e * (1 + 0.3 * np.exp(-(x**2 + y**2 + z**2) / (2 * 0.8**2))))
    for l in range(nl - 1):
        o.commup(l)
    vol0 = (12.0 / n) ** 3
    e0 = _composite_sum(o, nl, n, ENE, vol0)
    o.step(5)
    e1 = _composite_sum(o, nl, n, ENE, vol0)
    assert abs(e1 - e0) <= 1e-13 * abs(e0)


# ---------------------------------------------------------------- T3

@pytest.mark.parametrize("rho_u", [1.0, 2.0])
def test_diffusion_fourier_mode_exact(rho_u):
    """Explicit diffusion (Eqs. 19-22, sign fixed by Eq. 28): a Fourier mode of e/rho
    is multiplied per step by 1 - 4 chi dt sum_d sin^2(k_d dx_d/2)/dx_d^2."""
    n = (16, 12, 8)
    half = (2.0, 3.0, 1.0)
    chi, dt = 0.7, 0.2 * 0.25**2 / 0.7
    o = make(1, n, half, GM=0.0, L=0.0, chi=chi, hydro_on=0, dt_fixed=dt,
             bc=(I.BC_PERIODIC,) * 6, rho0=rho_u)
    lo, hi = tuple(-h for h in half), half
    x, y, z = centres(o, 0, n, lo, hi)
    m = (1, 2, 1)
    k = [2 * np.pi * m[d] / (hi[d] - lo[d]) for d in range(3)]
    dx = [(hi[d] - lo[d]) / n[d] for d in range(3)]
    e0 = o.get_field(0, ENE)[0, 0, 0]
    A = 0.05 * e0
    phase = k[0] * x + k[1] * y + k[2] * z
    o.set_field(0, ENE, e0 + A * np.cos(phase))
    steps = 7
    o.step(steps)
    g = 1 - 4 * chi * dt * sum(math.sin(k[d] * dx[d] / 2) ** 2 / dx[d] ** 2 for d in range(3))
    expect = e0 + A * g**steps * np.cos(phase)
    assert np.abs(o.get_field(0, ENE) - expect).max() <= 1e-12 * e0
    assert g**steps < 0.9  # the mode actually decayed


# ---------------------------------------------------------------- T4

def test_heat_kernel_variance_growth():
    """Heat kernel: the second moment of a diffusing bump grows as sigma0^2 + 2 chi t
    (exact for the conservative discrete Laplacian away from the boundary)."""
    n, half, chi = 48, 6.0, 1.0
    dt = 0.2 * 0.25**2 / chi
    o = make(1, n, half, GM=0.0, L=0.0, chi=chi, hydro_on=0, dt_fixed=dt,
             bc=(I.BC_PERIODIC,) * 6)
    x, y, z = centres(o, 0, n, (-half,) * 3, (half,) * 3)
    e0 = o.get_field(0, ENE)[0, 0, 0]
    s0 = 0.5
    bump = 0.1 * np.exp(-(x**2 + y**2 + z**2) / (2 * s0**2))
    o.set_field(0, ENE, e0 + bump)

    def moments():
        d = o.get_field(0, ENE) - e0
        return d.sum(), (d * x**2).sum() / d.sum(), d.max()

    M0, v0, p0 = moments()
    steps = 10
    o.step(steps)
    M1, v1, p1 = moments()
    t = steps * dt
    assert abs(M1 - M0) <= 1e-12 * M0
    assert abs((v1 - v0) - 2 * chi * t) <= 1e-9 * (2 * chi * t)
    # peak follows the analytic kernel (sigma0/sigma)^3 up to O(dx^2)
    s1 = math.sqrt(s0**2 + 2 * chi * t)
    assert abs(p1 / p0 - (s0 / s1) ** 3) < 0.03


def test_heat_kernel_second_order_convergence():
    """Heat kernel at a fixed time on 24^3 and 48^3 cells (dt proportional to dx^2):
    the largest deviation from the analytic Gaussian falls by ~4 when dx halves
    (second order in space; first order in time is O(dx^2) here too)."""
    half, chi, s0, T, amp = 6.0, 1.0, 1.0, 0.25, 0.1

    def max_error(n):
        dx = 2 * half / n
        dt = 0.2 * dx * dx / chi
        steps = int(round(T / dt))
        assert math.isclose(steps * dt, T)
        o = make(1, n, half, GM=0.0, L=0.0, chi=chi, hydro_on=0, dt_fixed=dt,
                 bc=(I.BC_PERIODIC,) * 6)
        x, y, z = centres(o, 0, n, (-half,) * 3, (half,) * 3)
        r2 = x**2 + y**2 + z**2
        e0 = o.get_field(0, ENE)[0, 0, 0]
        o.set_field(0, ENE, e0 + amp * np.exp(-r2 / (2 * s0**2)))
        o.step(steps)
        s1 = math.sqrt(s0**2 + 2 * chi * T)
        exact = amp * (s0 / s1) ** 3 * np.exp(-r2 / (2 * s1**2))
        return np.abs(o.get_field(0, ENE) - e0 - exact).max() / exact.max()

    coarse, fine = max_error(24), max_error(48)
    assert coarse < 0.03
    assert 3.5 < coarse / fine < 4.5, (coarse, fine)


def test_heat_kernel_nested_spreads():
    """Nested variant: a bump crossing level frontiers spreads as sigma^2 + 2 chi t."""
    n, nl, half, chi = 24, 3, 6.0, 0.2
    o = make(nl, n, half, GM=0.0, L=0.0, chi=chi, hydro_on=0, bc=(I.BC_PERIODIC,) * 6)
    s0 = 0.6
    for l in range(nl):
        x, y, z = centres(o, l, n, (-half,) * 3, (half,) * 3)
        e = o.get_field(l, ENE)
        o.set_field(l, ENE, e + 0.1 * np.exp(-(x**2 + y**2 + z**2) / (2 * s0**2)))
    for l in range(nl - 1):
        o.commup(l)
    e0 = I.base_params()["cs"] ** 2 / (5 / 3 * 2 / 3)

    def var():
        num = den = 0.0
        for l in range(nl):
            x, y, z = centres(o, l, n, (-half,) * 3, (half,) * 3)
            d = o.get_field(l, ENE) - e0
            w = np.ones_like(d, dtype=bool)
            if l < nl - 1:
                q = n // 4
                w[q:q + n // 2, q:q + n // 2, q:q + n // 2] = False
            vol = (2 * half / n / 2**l) ** 3
            num += (d * x**2)[w].sum() * vol
            den += d[w].sum() * vol
        return num / den

    v0 = var()
    o.step(10)
    grow = var() - v0
    assert abs(grow - 2 * chi * o.t) < 0.02 * (2 * chi * o.t)


# ---------------------------------------------------------------- T5 / T6

def _dispersion_roots(k, cs, chi, gamma):
    """Roots in omega of the denominator of Eq. 34 (rho_p = 0):
    i w (cs^2 - w^2/k^2) + chi (w^2 - k^2 cs^2/gamma) = 0, times i k^2."""
    return np.roots([1.0, 1j * chi * k**2, -(cs**2) * k**2, -1j * chi * cs**2 * k**4 / gamma])


def _mode(o, field, x, k):
    d = o.get_field(0, field)
    d = d - d.mean()
    return complex((d * np.cos(k * x)).sum(), (d * np.sin(k * x)).sum()) * 2 / d.size


def _linear_solution(k, chi, gamma, rho0, p0, t, y0):
    """Exact evolution of one Fourier mode exp(ikx) of the linearised Eqs. 26-28
    (no perturber): y = (rho, v_x, p) amplitudes; Eq. 34 is its dispersion relation."""
    from scipy.linalg import expm
    M = np.array([[0, -1j * rho0 * k, 0],
                  [0, 0, -1j * k / rho0],
                  [(p0 / rho0) * chi * k**2, -1j * gamma * p0 * k, -chi * k**2]], dtype=complex)
    return expm(M * t) @ np.asarray(y0, dtype=complex)


def _wave_run(chi, kind, steps, axis=0):
    nn, hh = [4, 4, 4], [0.5, 0.5, 0.5]
    nn[axis], hh[axis] = 32, 4.0
    n, half = tuple(nn), tuple(hh)
    gamma = 5 / 3
    o = make(1, n, half, GM=0.0, L=0.0, chi=chi, mach=0.0, bc=(I.BC_PERIODIC,) * 6)
    x = centres(o, 0, n, tuple(-h for h in half), half)[axis]
    xf = x - 0.125  # lower faces along the wave axis
    k = 2 * np.pi / 8.0
    A = 1e-5
    rho, e = o.get_field(0, RHO), o.get_field(0, ENE)
    p0 = (gamma - 1) * e[0, 0, 0]
    if kind == "isobaric":   # entropy (thermal) perturbation: delta p = 0, v = 0
        y0 = [-A, 0.0, 0.0]
        o.set_field(0, RHO, rho * (1 - A * np.cos(k * x)))
    else:                    # adiabatic sound wave travelling towards +axis
        y0 = [A, A, gamma * p0 * A]
        o.set_field(0, RHO, rho * (1 + A * np.cos(k * x)))
        o.set_field(0, ENE, e * (1 + gamma * A * np.cos(k * x)))
        o.set_field(0, VX + axis, A * np.cos(k * xf))
    out = []
    for _ in range(steps):
        o.step(25)
        z = _mode(o, RHO, x, k)
        y = _linear_solution(k, chi, gamma, 1.0, p0, o.t, y0)
        out.append((o.t, z, complex(y[0].real, -y[0].imag), k))
    return out, _dispersion_roots(k, 1.0, chi, gamma)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("chi", [0.05, 0.5])
def test_isobaric_mode_follows_linear_theory(chi, axis):
    """Thermal (isobaric) mode of the linearised Eqs. 26-28, whose slow root is the
    chi k^2 / gamma pole of Eq. 43: the density mode follows the exact linear
    solution within the O((k dx)^2) truncation error."""
    out, roots = _wave_run(chi, "isobaric", 10, axis)
    for t, z, y, _ in out:
        assert abs(abs(z) / abs(y) - 1) < 5e-3, (t, abs(z), abs(y))
    assert abs(out[-1][1]) < abs(out[0][1])


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("chi", [0.0, 0.3])
def test_sound_wave_follows_linear_theory(chi, axis):
    """Adiabatic sound wave (Eq. 35 for chi = 0; Eq. 34 with diffusion): amplitude
    and phase of the density mode follow the exact linear solution, so the wave
    travels at the acoustic root of Eq. 34."""
    out, roots = _wave_run(chi, "sound", 8, axis)
    ac = roots[np.argmax(roots.real)]
    for t, z, y, k in out:
        assert abs(abs(z) / abs(y) - 1) < 0.02, (t, abs(z), abs(y))
        # phase lag relative to the accumulated phase: speed within 0.5 %
        dph = np.angle(z / y)
        assert abs(dph) < 5e-3 * ac.real * t, (t, dph)
    t, z, _, k = out[-1]
    assert t * ac.real / k > 1.0  # the wave travelled more than one length unit


# ---------------------------------------------------------------- T7

def test_force_matches_brute_force_sum():
    """Eq. 18 summed level by level with covered coarse cells excluded equals a
    brute-force direct sum whose covered mask is built from physical coordinates."""
    n, nl, half = 24, 3, 6.0
    GM, eps = 0.013, 0.1
    o = make(nl, n, half, GM=GM, eps=eps)
    rng = np.random.default_rng(3)
    dens = []
    for l in range(nl):
        r = 1.0 + 0.05 * rng.standard_normal((n, n, n))
        o.set_field(l, RHO, r)
        dens.append(r)
    F = o.force()
    Fb = np.zeros(3, dtype=np.longdouble)
    for l in range(nl):
        x, y, z = centres(o, l, n, (-half,) * 3, (half,) * 3)
        h = half / 2**l
        vol = np.longdouble((2 * h / n) ** 3)
        cov = np.zeros_like(x, dtype=bool)
        if l < nl - 1:
            hc = h / 2
            cov = (np.abs(x) < hc) & (np.abs(y) < hc) & (np.abs(z) < hc)
        X, Y, Z = (a.astype(np.longdouble) for a in (x, y, z))
        r2 = X * X + Y * Y + Z * Z + np.longdouble(eps) ** 2
        w = np.longdouble(GM) * (dens[l].astype(np.longdouble) - 1) * vol / (r2 * np.sqrt(r2))
        w[cov] = 0
        Fb += np.array([(w * X).sum(), (w * Y).sum(), (w * Z).sum()])
    Fb = Fb.astype(np.float64)
    assert np.abs(F - Fb).max() <= 1e-12 * np.abs(Fb).max()
    # a density excess on +x pulls the perturber towards +x (attraction)
    o2 = make(1, 24, half, GM=GM, eps=eps)
    x, _, _ = centres(o2, 0, 24, (-half,) * 3, (half,) * 3)
    o2.set_field(0, RHO, 1.0 + 0.1 * (x > 1) * (x < 2))
    assert o2.force()[0] > 0


# ---------------------------------------------------------------- T8

def _element_positions(o, level, field, n, half, G):
    """positions of all elements of the padded array of one field"""
    dx = 2 * half / 2**level / n
    lo = -half / 2**level
    s = n + 2 * G
    idx = np.arange(s)
    cen = lo + (idx - G + 0.5) * dx
    face = lo + (idx - G) * dx
    axes = [cen, cen, cen]
    if field >= VX:
        axes[field - VX] = face
    z, y, x = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return x, y, z


def test_commup_reproduces_linear_fields():
    """CommUp (Fig. 2): a limited trilinear interpolation reproduces a linear field
    exactly on every fine ghost element, centred and staggered alike."""
    n, nl, half, G = 24, 2, 6.0, I.DEFAULT_G
    o = make(nl, n, half)
    coef = np.array([0.3, -0.7, 0.45, 1.1])
    for f in range(5):
        x, y, z = _element_positions(o, 0, f, n, half, G)
        o.set_full(0, f, coef[0] + 0.1 * f + coef[1] * x + coef[2] * y + coef[3] * z)
        o.set_full(1, f, np.full(x.shape, np.nan))
    o.commup(0)
    for f in range(5):
        x, y, z = _element_positions(o, 1, f, n, half, G)
        got = o.get_full(1, f)
        want = coef[0] + 0.1 * f + coef[1] * x + coef[2] * y + coef[3] * z
        ghost = np.ones(got.shape, dtype=bool)
        lo = [G, G, G]
        if f >= VX:  # both frontier faces of v_d come from the parent
            lo[2 - (f - VX)] = G + 1
        ghost[lo[0]:G + n, lo[1]:G + n, lo[2]:G + n] = False
        assert np.abs(got[ghost] - want[ghost]).max() < 1e-13, f
        assert np.isnan(got[~ghost]).all()  # active elements untouched


def test_commup_keeps_a_mirror_symmetric_state_symmetric():
    """CommUp of a state that is even in x (v_x odd) about the centre of the box
    gives fine ghosts with the same symmetry: the midway faces of v_x take the mean
    of their two coarse faces, and the two x frontier faces of v_x both come from
    the parent.  A one-sided reconstruction at the midway faces, or a lower
    frontier face left to the fine level, breaks it."""
    n, nl, half, G = 24, 2, 6.0, I.DEFAULT_G
    o = make(nl, n, half)
    rng = np.random.default_rng(11)
    s = n + 2 * G
    for f in range(5):
        r = rng.uniform(0.5, 1.5, (s, s, s))
        if f == VX:  # face I mirrors face s - I; face s/2 lies on the plane x = 0
            q = r.copy()
            q[:, :, 1:] = r[:, :, 1:] - r[:, :, :0:-1]
        else:  # cell I mirrors cell s - 1 - I
            q = 0.5 * (r + r[:, :, ::-1])
        o.set_full(0, f, q)
        o.set_full(1, f, rng.uniform(0.5, 1.5, (s, s, s)))
    o.commup(0)
    for f in range(5):
        a = o.get_full(1, f)
        kept = np.zeros(a.shape, dtype=bool)
        kept[G:G + n, G:G + n, (G + 1 if f == VX else G):G + n] = True
        if f == VX:
            filled = ~kept[:, :, 1:] & ~kept[:, :, :0:-1]
            d = np.abs(a[:, :, 1:] + a[:, :, :0:-1])[filled]
        else:
            filled = ~kept & ~kept[:, :, ::-1]
            d = np.abs(a - a[:, :, ::-1])[filled]
        assert d.size > 0 and d.max() == 0.0, (f, d.max())


def test_commup_is_bounded_by_neighbours():
    """van Leer-limited interpolation creates no new extrema."""
    n, nl, half, G = 24, 2, 6.0, I.DEFAULT_G
    o = make(nl, n, half)
    rng = np.random.default_rng(7)
    s = n + 2 * G
    q = rng.uniform(0.5, 1.5, (s, s, s))
    o.set_full(0, RHO, q)
    o.commup(0)
    got = o.get_full(1, RHO)
    from scipy.ndimage import maximum_filter, minimum_filter
    hi, lo = maximum_filter(q, size=3), minimum_filter(q, size=3)
    off = n // 4
    for (k, j, i) in [(0, 0, 0), (3, G + 5, 1), (s - 1, s - 1, s - 1), (G - 1, G + 3, G + n)]:
        host = [G + off + (c - G) // 2 for c in (k, j, i)]
        v = got[k, j, i]
        assert lo[tuple(host)] - 1e-15 <= v <= hi[tuple(host)] + 1e-15


def test_commmean_averages_linear_fields_in_band():
    """CommMean (Figs. 3-4): centred coarse cells take the mean of 8 fine cells and
    staggered faces the mean of 4 coplanar fine faces -- exact for linear fields --
    and only the band of coarse cells along the inner contour is overwritten."""
    n, nl, half, G = 24, 2, 6.0, I.DEFAULT_G
    band = 3
    o = make(nl, n, half, band=band)
    coef = np.array([0.2, 0.5, -0.3, 0.8])
    s = n + 2 * G
    for f in range(5):
        x, y, z = _element_positions(o, 1, f, n, half, G)
        o.set_full(1, f, coef[0] + coef[1] * x + coef[2] * y + coef[3] * z + f)
        o.set_full(0, f, np.full((s, s, s), -99.0))
    o.commmean(0)
    q, w = n // 4, n // 2
    a = np.arange(n)
    for f in range(5):
        x, y, z = _element_positions(o, 0, f, n, half, G)
        got = o.get_full(0, f)[G:G + n, G:G + n, G:G + n]
        want = (coef[0] + coef[1] * x + coef[2] * y + coef[3] * z + f)[G:G + n, G:G + n, G:G + n]
        # independent band mask: distance (in coarse cells) to the covered box edge
        dist = np.minimum(a - q, q + w - 1 - a)
        D = [dist, dist, dist]
        inside = [(a >= q) & (a < q + w)] * 3
        zz, yy, xx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        cov = inside[0][xx] & inside[1][yy] & inside[2][zz]
        dmin = np.minimum(np.minimum(D[0][xx], D[1][yy]), D[2][zz])
        cell_band = cov & (dmin < band)
        if f < 2:
            mask = cell_band
        else:
            ax = f - VX
            cc = [xx, yy, zz]
            lower = [c.copy() for c in cc]
            lower[ax] = lower[ax] - 1
            ok = (cc[ax] > q) & (cc[ax] < q + w)
            in_lower = np.zeros_like(cell_band)
            valid = (lower[ax] >= 0)
            in_lower[valid] = cell_band[lower[2][valid], lower[1][valid], lower[0][valid]]
            mask = cov & ok & (cell_band | in_lower)
        assert np.abs(got[mask] - want[mask]).max() < 1e-13, f
        assert (got[~mask] == -99.0).all(), f
        assert mask.sum() > 0


# ---------------------------------------------------------------- T9

def test_xi_search_appendix_cases():
    rows = []
    with open(os.path.join(GOLDEN, "xi_search_appendix_a.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if not line:
                continue
            a, b, c = (part.split() for part in line.split(";"))
            rows.append(([float(v) for v in a], [float(v) for v in b], [int(v) for v in c]))
    assert len(rows) >= 8
    for dtl, cost, want in rows:
        _, xi = xi_search(dtl, cost)
        assert xi == want, (dtl, xi, want)


# ---------------------------------------------------------------- T10

@pytest.mark.parametrize("av", [0.0, 2.0])
def test_ghost_and_band_width_sufficient(av):
    """Widening the ghost buffer (Sec. 3.2.1) or the CommMean band (Sec. 3.2.2) leaves
    every active cell -- and the force -- bitwise unchanged, with and without the
    artificial viscosity."""
    n, nl, half = 24, 3, 6.0

    def run(G, band):
        o = make(nl, n, half, G=G, band=band, GM=0.01, eps=0.25, L=0.05, lum_sigma=0.25,
                 av_c2=av)
        _perturb(o, nl, n, seed=11)
        if av:
            for l in range(nl):  # strong enough to compress: the viscosity acts
                v = o.get_field(l, VX)
                o.set_field(l, VX, v - 0.4 * np.sin(2 * np.pi * np.arange(n) / n)[None, None, :])
            for l in range(nl - 1):
                o.commup(l)
        o.step(3)
        out = []
        for l in range(nl):
            a = np.stack([o.get_field(l, f) for f in range(5)])
            if l < nl - 1:
                q = n // 4
                a[:, q:q + n // 2, q:q + n // 2, q:q + n // 2] = 0
            out.append(a)
        return out, o.force()

    ref, Fr = run(I.DEFAULT_G, I.DEFAULT_BAND)
    for G, band in [(I.DEFAULT_G + 2, I.DEFAULT_BAND), (I.DEFAULT_G, I.DEFAULT_BAND + 1)]:
        got, F = run(G, band)
        for l in range(nl):
            assert np.array_equal(got[l], ref[l]), (G, band, l)
        assert np.array_equal(F, Fr)


# ---------------------------------------------------------------- sources

@pytest.mark.parametrize("sigma", [0.0, 0.5])
def test_luminosity_deposit_total(sigma):
    """The energy L dt is deposited in full each level step (Sec. 3.4)."""
    n, half, L = 16, 2.0, 0.37
    dt = 1e-3
    o = make(1, n, half, GM=0.0, L=L, lum_sigma=sigma, chi=0.0, hydro_on=0, dt_fixed=dt,
             bc=(I.BC_PERIODIC,) * 6)
    vol = (2 * half / n) ** 3
    E0 = o.get_field(0, ENE).sum() * vol
    o.step(5)
    E1 = o.get_field(0, ENE).sum() * vol
    assert abs((E1 - E0) - 5 * L * dt) < 1e-12 * E0
    d = o.get_field(0, ENE) - o.get_field(0, ENE).min()
    if sigma == 0.0:
        assert (d > 0).sum() == 8  # the eight cells sharing the vertex at the origin
        assert np.allclose(d[d > 0], d[d > 0][0], rtol=0, atol=1e-14)


def test_gaussian_luminosity_profile():
    """The Gaussian deposit (reading R10): per level step every active cell gains
    energy in proportion to exp(-r_c^2 / (2 sigma^2)) of its centre; the total is
    L dt."""
    n, half, L, sigma, dt = 16, 2.0, 0.37, 0.6, 1e-3
    o = make(1, n, half, GM=0.0, L=L, lum_sigma=sigma, chi=0.0, hydro_on=0, dt_fixed=dt,
             bc=(I.BC_PERIODIC,) * 6)
    e0 = o.get_field(0, ENE).copy()
    o.step(1)
    d = o.get_field(0, ENE) - e0
    x, y, z = centres(o, 0, n, (-half,) * 3, (half,) * 3)
    r2 = (x**2 + y**2 + z**2).ravel()
    dv = d.ravel()
    assert np.all(dv > 0)
    # log d + r^2/(2 sigma^2) is one constant; a wrong width, centre or power of r
    # leaves a trend.  Each increment is a difference of energies ~1 apart from it,
    # so its relative rounding error is a few ulps of e / d.
    c = np.log(dv) + r2 / (2 * sigma**2)
    tol = 8 * np.finfo(float).eps * np.abs(o.get_field(0, ENE)).ravel() / dv
    ref = int(np.argmax(dv))
    assert np.all(np.abs(c - c[ref]) <= tol + tol[ref]), np.max(np.abs(c - c[ref]) / tol)
    assert d.sum() * (2 * half / n) ** 3 == pytest.approx(L * dt, rel=1e-12)


def test_entropy_wave_advection_converges():
    """An entropy wave (density varies, pressure and velocity uniform) is carried by
    the wind unchanged (Eqs. 1-3 with GM = L = chi = 0).  After one crossing of a
    periodic box, pressure and velocity stay uniform to O(a^2), and the rms density
    error falls by ~2^1.75 when dx halves: van Leer's limiter clips the extrema, so
    the order lies between 1.5 and 2 (a first-order scheme gives 2^1)."""
    a, Lx, mach = 1e-3, 4.0, 1.0
    lo, hi = (-Lx / 2, -0.5, -0.5), (Lx / 2, 0.5, 0.5)
    k = 2 * math.pi / Lx

    def rms_error(n):
        dx = Lx / n
        x = lo[0] + (np.arange(n) + 0.5) * dx
        avg = 1 + a * (np.cos(k * (x - dx / 2)) - np.cos(k * (x + dx / 2))) / (k * dx)
        T = Lx / (mach * 1.0)
        steps = int(math.ceil(T / (0.4 * dx / (1 + mach))))
        p = I.base_params(GM=0.0, L=0.0, chi=0.0, mach=mach, flow_dir=(1.0, 0.0, 0.0),
                          bc=(I.BC_PERIODIC,) * 6, dt_fixed=T / steps)
        o = Oracle(1, (n, 8, 8), lo, hi, I.DEFAULT_G, p)
        e0 = o.get_field(0, ENE)[0, 0, 0]
        o.set_field(0, RHO, np.broadcast_to(avg, (8, 8, n)).copy())
        o.step(steps)
        assert math.isclose(o.t, T)
        assert np.abs(o.get_field(0, ENE) - e0).max() < 1e-5 * a
        assert np.abs(o.get_field(0, VX) - mach).max() < 1e-5 * a
        r = o.get_field(0, RHO)
        assert np.abs(r - r[:1, :1, :]).max() < 1e-14  # still one-dimensional
        return math.sqrt(((r[0, 0] - avg) ** 2).mean()) / a

    e32, e64 = rms_error(32), rms_error(64)
    assert e32 < 0.04
    assert 2.8 < e32 / e64 < 4.2, (e32, e64)


def test_gravity_kick_points_to_perturber():
    """First-order check of S (Eq. 15) with the attractive Plummer potential:
    a gas at rest acquires v = -dt grad Phi, Phi = -GM/sqrt(r^2+eps^2)."""
    n, half, GM, eps = 16, 4.0, 1.0, 0.5
    dt = 1e-5
    o = make(1, n, half, GM=GM, eps=eps, mach=0.0, chi=0.0, dt_fixed=dt,
             bc=(I.BC_OUTFLOW,) * 6)
    o.step(1)
    x, y, z = centres(o, 0, n, (-half,) * 3, (half,) * 3)
    xf = x - 0.25
    vx = o.get_field(0, VX)
    r2 = xf**2 + y**2 + z**2 + eps**2
    ax = -GM * xf / r2**1.5
    sel = (np.abs(xf) > 1.0) & (np.abs(xf) < 3.0) & (np.abs(y) < 1.5) & (np.abs(z) < 1.5)
    ratio = vx[sel] / (ax[sel] * dt)
    assert np.all(np.abs(ratio - 1) < 0.05)


# ---------------------------------------------------------------- momentum

@pytest.mark.parametrize("av", [0.0, 2.0])
def test_momentum_conserved_periodic(av):
    """Without gravity, the pressure kick, the artificial viscosity (a difference of
    viscous pressures across each face) and the flux-form momentum transport keep
    sum_faces rho_face v (each component) constant in a periodic box."""
    n = 16
    o = make(1, n, 4.0, GM=0.0, L=0.0, chi=0.2, mach=0.6, flow_dir=(0.36, 0.48, 0.8),
             bc=(I.BC_PERIODIC,) * 6, av_c2=av)
    _perturb(o, 1, n, seed=21, amp=3e-2 if av == 0 else 0.3)
    G = I.DEFAULT_G

    def momentum():
        rho = o.get_full(0, RHO)
        out = []
        for m in range(3):
            v = o.get_full(0, VX + m)
            ax = 2 - m  # numpy axis of coordinate m
            rl = np.roll(rho, 1, axis=ax)
            pm = 0.5 * (rl + rho) * v
            out.append(pm[G:G + n, G:G + n, G:G + n].sum())
        return np.array(out)

    o.fill_bc()
    P0 = momentum()
    o.step(5)
    o.fill_bc()
    P1 = momentum()
    assert np.abs(P1 - P0).max() < 1e-13 * n**3


def test_nested_momentum_drift_is_bounded():
    """Across a level frontier the staggered momenta are not flux-matched (only mass and
    energy are, Sec. 3.2.3), so the coarse level's momentum, conserved by its own solver
    in a periodic box, moves when CommMean restricts the covered faces.  This states by
    how much, from the first coarse step on (when the covered cells first hold the
    restriction), beside the composite mass, which stays exact."""
    n, nl = 24, 2
    o = make(nl, n, 6.0, GM=0.0, L=0.0, chi=0.3, mach=0.8, flow_dir=(0.6, 0.8, 0.0),
             bc=(I.BC_PERIODIC,) * 6)
    _perturb(o, nl, n, seed=5)
    G = I.DEFAULT_G
    vol0 = (12.0 / n) ** 3

    def momentum():
        o.fill_bc()
        rho = o.get_full(0, RHO)
        P, S = [], []
        for m in range(3):
            v = o.get_full(0, VX + m)
            pm = 0.5 * (np.roll(rho, 1, axis=2 - m) + rho) * v
            P.append(pm[G:G + n, G:G + n, G:G + n].sum() * vol0)
            S.append(np.abs(pm[G:G + n, G:G + n, G:G + n]).sum() * vol0)
        return np.array(P), np.array(S)

    o.step(1)
    P0, S0 = momentum()
    m0 = _composite_sum(o, nl, n, RHO, vol0)
    o.step(4)
    P1, _ = momentum()
    m1 = _composite_sum(o, nl, n, RHO, vol0)
    drift = np.abs(P1 - P0) / S0
    print("momentum drift / sum |rho v| per component after 4 coarse steps:", drift)
    assert abs(m1 - m0) <= 1e-13 * abs(m0)
    assert drift.max() < 2e-3


@pytest.mark.parametrize("adv,comp", [(0, 1), (1, 2), (2, 0)])
def test_transverse_momentum_advected_at_wind_speed(adv, comp):
    """A shear wave v_comp(x_adv) in a uniform wind along x_adv is carried
    at the wind speed (transport of a staggered component across its edges)."""
    nn, hh = [4, 4, 4], [0.5, 0.5, 0.5]
    nn[adv], hh[adv] = 32, 4.0
    fd = [0.0, 0.0, 0.0]
    fd[adv] = 1.0
    U = 0.3
    o = make(1, tuple(nn), tuple(hh), GM=0.0, L=0.0, chi=0.0, mach=U, flow_dir=tuple(fd),
             bc=(I.BC_PERIODIC,) * 6)
    x = centres(o, 0, tuple(nn), tuple(-h for h in hh), tuple(hh))[adv]
    k = 2 * np.pi / 8.0
    A = 1e-3
    o.set_field(0, VX + comp, A * np.sin(k * x))
    z0 = _mode(o, VX + comp, x, k)
    o.step(100)
    z1 = _mode(o, VX + comp, x, k)
    shift = np.angle(z1 / z0) / k  # distance travelled by the pattern
    assert abs(shift - U * o.t) < 0.01 * U * o.t
    assert 0.9 < abs(z1) / abs(z0) <= 1.0


# ---------------------------------------------------------------- T11

def _ostriker_subsonic(mach):
    """Linear-theory drag factor of a subsonic perturber (Ostriker 1999, the adiabatic
    force F_adi = F0 M^-2 I the paper quotes as Eq. 54), valid once c_s t > r_min/(1-M)."""
    return 0.5 * math.log((1 + mach) / (1 - mach)) - mach


def test_adiabatic_subsonic_drag_approaches_linear_theory():
    """chi = 0, L = 0, Mach 0.5, weak perturber (GM well below the finest cell): the
    force along the motion settles near -F0 I / M^2 (Eqs. 50, 54) while the sound
    sphere is still inside the box."""
    M, GM, nl, n, half = 0.5, 0.01, 4, 32, 16.0
    dxf = 2 * half / n / 2 ** (nl - 1)
    o = make(nl, n, half, mach=M, GM=GM, chi=0.0, L=0.0, eps=2 * dxf)
    F0 = 4 * math.pi * GM**2  # rho0 = c_s = 1
    Fth = -F0 * _ostriker_subsonic(M) / M**2
    ratios = []
    while o.t < 7.0:
        o.step(4)
        ratios.append((o.t, o.force()[0] / Fth))  # the perturber moves along +x
    late = [r for t, r in ratios if 3.5 < t < 7.0]
    assert late and all(0.95 < r < 1.06 for r in late), ratios
