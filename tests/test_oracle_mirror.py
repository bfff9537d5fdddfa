"""Mirror planes (the quadrant domain of Sec. 3.4): a run on the part x > 0 (and
y > 0) of the domain, with reflecting walls on the planes through the perturber,
must reproduce that part of the run on the whole domain, the force of the whole
domain included.  The whole-domain run uses none of the mirror logic, so this pins
every piece of it (the ghost fill of finer levels, CommUp across the plane, the
frontier and band rules, the luminosity weights, the force multiplicity) against
the unfolded problem.  Oracle only (CPU)."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1812_03191_gb300 import inputs as I

R, E, VX, VY, VZ = range(5)
HALF = 3.0
N = 24


def _params(mirror, **over):
    bc = [I.BC_REFLECT] * 4 + [I.BC_INFLOW, I.BC_OUTFLOW]
    if not mirror[1]:
        bc[2] = bc[3] = I.BC_OUTFLOW
    p = I.base_params(gamma=1.4, mach=0.8, flow_dir=(0.0, 0.0, 1.0), GM=0.05, eps=0.0,
                      chi=0.3, L=0.02, lum_sigma=0.0, bc=tuple(bc))
    p.update(over)
    return p


def _pair(n_levels, mirror, **over):
    p = _params(mirror, **over)
    full = Oracle(n_levels, N, (-HALF,) * 3, (HALF,) * 3, I.DEFAULT_G, p)
    n = tuple(N // 2 if m else N for m in mirror) + (N,)
    lo = tuple(0.0 if m else -HALF for m in mirror) + (-HALF,)
    part = Oracle(n_levels, n, lo, (HALF,) * 3, I.DEFAULT_G, p)
    return full, part


def _part_of(a, mirror):
    """the x > 0 (and y > 0) part of a whole-domain field (z, y, x order)"""
    if mirror[0]:
        a = a[:, :, N // 2:]
    if mirror[1]:
        a = a[:, N // 2:, :]
    return a


MIRRORS = [(True, True), (True, False)]


@pytest.mark.parametrize("mirror", MIRRORS, ids=["quadrant", "half"])
@pytest.mark.parametrize("n_levels,over", [
    (1, {}),
    (2, {}),
    (3, dict(xi_mode=1)),
    (2, dict(lum_sigma=0.3, av_c2=1.0)),
], ids=["1level", "2levels", "3levels_xi", "2levels_gauss_visc"])
def test_mirrored_run_reproduces_the_unfolded_domain(mirror, n_levels, over):
    full, part = _pair(n_levels, mirror, **over)
    for _ in range(3):
        full.step(4)
        part.step(4)
        assert part.last_dt == pytest.approx(full.last_dt, rel=1e-13)
    for l in range(n_levels):
        for f in range(5):
            a = _part_of(full.get_field(l, f), mirror)
            b = part.get_field(l, f)
            bg = {R: 1.0, E: full.get_field(l, E).max()}.get(f, 1.0)
            assert np.abs(a - b).max() <= 1e-12 * bg, (l, f, np.abs(a - b).max())
    # the state has moved away from the background by much more than the tolerance
    assert np.abs(part.get_field(n_levels - 1, R) - 1.0).max() > 1e-3
    Ff, Fp = full.force(), part.force()
    assert abs(Ff[2]) > 1e-4
    assert Fp[2] == pytest.approx(Ff[2], rel=1e-11)
    assert Fp[0] == 0.0 and abs(Ff[0]) < 1e-11 * abs(Ff[2])
    if mirror[1]:
        assert Fp[1] == 0.0 and abs(Ff[1]) < 1e-11 * abs(Ff[2])
    else:
        assert Fp[1] == pytest.approx(Ff[1], rel=1e-9, abs=1e-12 * abs(Ff[2]))


def test_mirrored_run_keeps_the_wall_velocity_at_zero():
    """v_x on the plane x = 0 stays zero on every level (no mass crosses a mirror)"""
    _, part = _pair(2, (True, True))
    part.step(8)
    for l in range(2):
        assert np.abs(part.get_field(l, VX)[:, :, 0]).max() == 0.0
        assert np.abs(part.get_field(l, VY)[:, 0, :]).max() == 0.0


def test_child_on_the_plane_needs_a_mirror():
    """a finer level may start on the domain's lower face only across a mirror plane"""
    p = _params((True, True), bc=(I.BC_OUTFLOW,) + (I.BC_REFLECT,) * 3 + (I.BC_INFLOW,) * 2)
    with pytest.raises(ValueError):
        Oracle(2, (12, 12, 24), (0.0, 0.0, -HALF), (HALF,) * 3, I.DEFAULT_G, p)
    Oracle(1, (12, 12, 24), (0.0, 0.0, -HALF), (HALF,) * 3, I.DEFAULT_G, p).close()
