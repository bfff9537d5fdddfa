"""Pins of the level-0 boundary fill (Sec. 3.4 set-up: injection and outflow faces,
symmetric walls) against the mirror symmetry of the problem.

The perturber sits at the centre of a box whose faces are all of one type, or in a
wind along x: the problem is then symmetric under y -> -y and z -> -z (and, at rest,
under every reflection), so the discrete solution must be too, whatever the fill
does elsewhere.  A fill that treats the lower and the upper boundary face of the
staggered normal velocity differently breaks that symmetry and gives the perturber
a spurious transverse force.  CPU only.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_1812_03191_gb300 import inputs as I

RHO, ENE, VX, VY, VZ = range(5)


def make(nl, n, half, **over):
    return Oracle(nl, n, (-half,) * 3, (half,) * 3, I.DEFAULT_G, I.base_params(**over))


def force_scale(o, nl, n, half, GM, eps):
    """sum over the active cells of every level of |each term of Eq. 18|: the size of
    the force's rounding error, whatever the summation order"""
    s = 0.0
    for l in range(nl):
        h = half / 2**l
        dx = 2 * h / n
        ax = -h + (np.arange(n) + 0.5) * dx
        z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
        r2 = x * x + y * y + z * z + eps * eps
        w = GM * np.abs(o.get_field(l, RHO) - 1.0) * dx**3 / (r2 * np.sqrt(r2))
        s += float((w * np.sqrt(x * x + y * y + z * z)).sum())
    return s


@pytest.mark.parametrize("bc", [I.BC_OUTFLOW, I.BC_INFLOW])
@pytest.mark.parametrize("nl", [1, 2])
def test_perturber_at_rest_feels_no_force(bc, nl):
    """At rest in a box with the same boundary type on all six faces the wake is
    spherical: every component of Eq. 18 vanishes to rounding."""
    n, half, GM, eps = 24, 6.0, 0.01, 0.5
    o = make(nl, n, half, mach=0.0, GM=GM, eps=eps, chi=1.0, bc=(bc,) * 6)
    o.step(10)
    F = o.force()
    S = force_scale(o, nl, n, half, GM, eps)
    assert S > 1e-8  # the gas did respond to the perturber
    assert np.abs(F).max() <= 1e-13 * S, (F, S)


def _check_mirror(o, level, exact):
    """y -> -y and z -> -z symmetry of the active cells: rho, e, v_x even, v_y odd
    in y (faces j and n - j mirror each other; face 0 has no partner among the
    active elements), v_z odd in z"""
    tol = 0 if exact else 4 * np.finfo(float).eps
    f = [o.get_field(level, k) for k in range(5)]
    for ax in (1, 0):  # numpy axes of y and z (fields are (nz, ny, nx))
        for k in (RHO, ENE, VX):
            a = f[k]
            ref = np.abs(a).max() if k < 2 else 1.0
            assert np.abs(a - np.flip(a, axis=ax)).max() <= tol * ref, (level, ax, k)
        odd = f[VY] if ax == 1 else f[VZ]
        even = f[VZ] if ax == 1 else f[VY]
        inner = np.take(odd, np.arange(1, odd.shape[ax]), axis=ax)
        assert np.abs(inner + np.flip(inner, axis=ax)).max() <= tol, (level, ax)
        assert np.abs(even - np.flip(even, axis=ax)).max() <= tol, (level, ax)


def test_wind_run_keeps_its_mirror_symmetry_bitwise():
    """One level, Mach 0.5 wind along -x, injection at +x, outflow elsewhere: the
    transverse mirror symmetry holds bit for bit (each operator's arithmetic is
    mirror-exact: differences, negations and commutative sums)."""
    n, half = 24, 6.0
    o = make(1, n, half, GM=0.01, eps=0.5, chi=1.0, L=0.05, lum_sigma=0.5)
    o.step(12)
    _check_mirror(o, 0, exact=True)
    # the force sum runs in index order, which a reflection does not keep: the
    # transverse components are rounding residues of the sum
    F = o.force()
    S = force_scale(o, 1, n, half, 0.01, 0.5)
    assert F[0] < 0 and np.abs(F[1:]).max() <= 1e-13 * S, (F, S)


def test_nested_wind_run_keeps_its_mirror_symmetry():
    """Three levels: the frontier flux sums (Sec. 3.2.3) add the fine faces in a fixed
    order, which a reflection permutes, so the symmetry holds to a few ulp; the
    transverse force is a rounding residue of the drag."""
    n, half, nl = 24, 6.0, 3
    o = make(nl, n, half, GM=0.01, eps=0.25, chi=1.0, L=0.05, lum_sigma=0.25)
    o.step(8)
    for l in range(nl):
        _check_mirror(o, l, exact=False)
    F = o.force()
    assert np.abs(F[1:]).max() <= 1e-12 * abs(F[0]), F


def _injection_run(upper):
    n, half, G = 16, 4.0, I.DEFAULT_G
    sgn = -1.0 if upper else 1.0
    bc = [I.BC_OUTFLOW] * 6
    bc[1 if upper else 0] = I.BC_INFLOW
    o = make(1, n, half, mach=0.7, flow_dir=(sgn, 0.0, 0.0), GM=0.02, eps=0.5, chi=1.0,
             bc=tuple(bc))
    o.step(6)
    return o, n, G, sgn


@pytest.mark.parametrize("upper", [False, True])
def test_injection_face_holds_the_wind_velocity(upper):
    """The fill sets an injection (inflow) face's boundary face of v_x to the
    background V, on a lower face (wind along +x, injection at -x) as on an upper
    one (wind along -x, injection at +x)."""
    o, n, G, sgn = _injection_run(upper)
    face = G + n if upper else G
    moved = np.abs(o.get_full(0, VX)[G:G + n, G:G + n, face] - sgn * 0.7).max()
    assert moved > 1e-6  # the solver moved it during the steps
    o.fill_bc()
    assert np.all(o.get_full(0, VX)[:, :, face] == sgn * 0.7)


def test_injection_through_a_lower_or_an_upper_face_are_mirror_images():
    """The run with injection at -x is the mirror image under x -> -x of the run with
    injection at +x, bit for bit: rho, e, v_y, v_z even, v_x odd (face i of one is
    face n - i of the other)."""
    a, n, G, _ = _injection_run(False)
    b, _, _, _ = _injection_run(True)
    for k in (RHO, ENE, VY, VZ):
        fa, fb = a.get_field(0, k), b.get_field(0, k)
        assert np.array_equal(fa, fb[:, :, ::-1]), k
    va = a.get_full(0, VX)[G:G + n, G:G + n, G:G + n + 1]
    vb = b.get_full(0, VX)[G:G + n, G:G + n, G:G + n + 1]
    assert np.array_equal(va, -vb[:, :, ::-1])


def test_outflow_boundary_faces_evolve_alike():
    """Under outflow both boundary faces of v_x are left to the solver and the ghost
    faces beyond copy them: with the wind along y, the x-problem is symmetric, and the
    lower and upper boundary faces of v_x are each other's negatives."""
    n, half, G = 16, 4.0, I.DEFAULT_G
    o = make(1, n, half, mach=0.5, flow_dir=(0.0, -1.0, 0.0), GM=0.02, eps=0.5, chi=1.0,
             bc=(I.BC_OUTFLOW, I.BC_OUTFLOW, I.BC_OUTFLOW, I.BC_INFLOW, I.BC_OUTFLOW,
                 I.BC_OUTFLOW))
    o.step(6)
    vx = o.get_full(0, VX)[G:G + n, G:G + n]
    lo, hi = vx[:, :, G], vx[:, :, G + n]
    assert np.abs(lo).max() > 1e-8  # the faces moved
    assert np.array_equal(lo, -hi)
    # the fill leaves both boundary faces alone and copies each into the ghost faces
    # beyond it
    o.fill_bc()
    vf = o.get_full(0, VX)[G:G + n, G:G + n]
    assert np.array_equal(vf[:, :, G], lo) and np.array_equal(vf[:, :, G + n], hi)
    for g in range(1, G):
        assert np.array_equal(vf[:, :, G - g], lo) and np.array_equal(vf[:, :, G + n + g], hi)
