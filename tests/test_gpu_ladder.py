"""Heating force by differencing hot and cold runs (Eq. 5) over a ladder of nested
levels at Mach 3, with the paper's Sec. 4.1 set-up, run as pairs in one pool."""
import numpy as np
import pytest

from paper_1812_03191_gb300 import binding
from paper_1812_03191_gb300 import ladder

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1812_03191_gb300 import build as B
    B.build()
    binding.load()


def test_heating_force_grows_by_the_eq24_increment_per_level():
    """Each added level halves the finest cell and should raise the supersonic heating
    force by (gamma - 1) GM L ln2 / (chi V^2) (Eq. 24).  That is the asymptotic
    increment; at these resolutions (r_min V / 4 chi between 0.02 and 0.14) Eq. 10-12
    give 0.6-0.85 of it.  Measured (100 tau): 0.77-0.81 at every step of the ladder."""
    out = ladder.run(levels=(4, 5, 6), t_end_taus=30.0, sample_every=8)
    pred = out["predicted_increment"]
    fin = [out["runs"][nl]["final"] for nl in (4, 5, 6)]
    assert all(f > 0 for f in fin)  # a thrust along the motion (Sec. 4.1)
    inc = np.diff(fin)
    assert np.all(inc > 0.6 * pred) and np.all(inc < 1.0 * pred), (inc / pred)
    # the same increment at every step: the logarithmic law of Eq. 13
    assert abs(inc[1] - inc[0]) < 0.15 * pred, (inc / pred)
    # settled: the last quarter of each history moves by under 2 %
    for nl in (4, 5, 6):
        F = np.array(out["runs"][nl]["F_heating"])
        k = len(F)
        assert abs(F[-1] - F[3 * k // 4]) < 0.02 * abs(F[-1])


def test_low_mach_heating_force_matches_eq8_within_the_box_share():
    """Mach 0.1, 6 levels, 100 tau: the heating force equals Eq. 8 times the share
    h(r'_max) - h(r'_min) = 0.918 of Eq. 23 that the box and the finest cell hold
    (measured: within 0.6 %; the paper's Fig. 6 inset: within ~3 %)."""
    out = ladder.low_mach(mach=0.1)
    assert out["eq23_share"] == pytest.approx(0.918, abs=1e-3)
    assert abs(out["ratio"] - 1.0) < 0.03, out["ratio"]


@pytest.mark.parametrize("quadrant", [False, True], ids=["whole_box", "quadrant"])
def test_low_mach_cold_thermal_force_is_a_drag_of_the_eq51_order(quadrant):
    """Cold perturber with thermal diffusion minus the adiabatic one at Mach 0.1,
    6 levels, l = 100 lambda, 100 tau: a settled drag, as Sec. 4.2 finds, of the
    order of -(gamma - 1)/2 F0 (Eq. 51) times the Eq. 23 share.  It is the V -> 0
    limit, which the paper corroborates in a box 32 times larger and with its own
    boundaries (mirror walls, the background held on both faces along the flow):
    on the quadrant meshes with those boundaries the ratio must lie within
    0.8-1.05 (measured 1.03) with a settled second half.  The whole box has
    zero-gradient outflow on five faces, which the paper does not use: there the
    drag is still decaying at 100 tau (measured 0.76 of the value, from 1.02 at
    half the run), so only a drag of the same order is required."""
    out = ladder.cold_thermal(mach=0.1, quadrant=quadrant)
    print(f"cold thermal force, {'quadrant' if quadrant else 'whole box'}: ratio "
          f"{out['ratio']:.3f} of Eq. 51 x Eq. 23 share")
    F = np.array(out["runs"][6]["F"])
    late = F[len(F) // 2:]
    assert F[-1] < 0 and np.all(late < 0)  # a drag
    if quadrant:
        assert 0.8 < out["ratio"] < 1.05, out["ratio"]
        assert np.abs(late - F[-1]).max() <= 0.1 * abs(F[-1])  # settled
    else:
        assert 0.5 < out["ratio"] < 1.1, out["ratio"]


def test_cold_thermal_force_in_the_papers_geometry():
    """Sec. 4.2 in the geometry the paper uses for it: the quadrant domain with its
    mirror planes, a ground of 64 x 64 x 128 under levels of 32 x 32 x 64 (the first
    over a quarter of the ground), l = 3200 lambda, here 9 levels, Mach 0.1, 100 tau.
    The paper matches the V -> 0 value -(gamma - 1)/2 F0 to within a few per cent.
    Measured: 0.992 of it times the Eq. 23 share of this box and finest cell (0.993
    and 0.994 with 10 and 11 levels)."""
    out = ladder.paper_cold_thermal(n_levels=9)
    assert 0.97 < out["ratio"] < 1.03, out["ratio"]
    F = np.array(out["F"])
    assert F[-1] < 0 and np.abs(F[len(F) // 2:] - F[-1]).max() <= 0.1 * abs(F[-1])


def test_low_mach_heating_force_on_the_papers_quadrant_meshes():
    """The low-Mach heating force on the paper's own 16 x 16 x 32 quadrant meshes with
    their mirror planes (6 levels, l = 100 lambda): the same Eq. 8 x Eq. 23 value as
    the whole box (measured: 1.0027 here, 1.0021 there)."""
    out = ladder.low_mach(mach=0.1, quadrant=True)
    assert abs(out["ratio"] - 1.0) < 0.03, out["ratio"]

