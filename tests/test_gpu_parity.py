"""GPU (CUDA path through the C ABI) versus the FP64 oracle, element by element.

Tolerance (FP64 path): per field and level, max|gpu - oracle| / s_f <= 1e-10, with
s_f = 1 for rho and e and s_f = max(V, 1e-3 c_s) for the velocities.  The two sides
differ only in rounding order (the GPU contracts multiply-adds, the oracle does not;
the force sum is a tree on the GPU).

The force is linear in the density (Eq. 18), so its difference is bounded by the
density difference the field check measures: |dF_d| <= sum_c |w_c| |drho_c| +
rounding <= (max|drho| + 2 eps) sum_c |w_c| + N eps sum_c |w_c (rho_c - rho0)|, with
w_c = GM V_c r_c / (r^2 + eps_s^2)^1.5 over the uncovered active cells (2 eps: the
deviation the library sums and the full density the oracle stores each round once;
the last term: the oracle's sequential sum of N terms).  Each test checks that
bound, with no other slack, and prints the achieved relative force error.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_1812_03191_gb300 import binding
from paper_1812_03191_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1812_03191_gb300 import build as B
    B.build()
    binding.load()


TRANSPORTS = [binding.TRANSPORT_SEPARATE, binding.TRANSPORT_FUSED]
TRANSPORT_IDS = ["separate", "fused"]


def pair(nl, n, half, params, G=I.DEFAULT_G, precision=binding.DF_FP64,
         transport=binding.TRANSPORT_AUTO):
    lo = tuple(-h for h in half) if not np.isscalar(half) else (-half,) * 3
    hi = tuple(half) if not np.isscalar(half) else (half,) * 3
    sim = binding.Sim(nl, n, lo, hi, G, params, precision=precision)
    sim.set_transport(transport)
    orc = Oracle(nl, n, lo, hi, G, params)
    return sim, orc


def field_errors(sim, orc, params):
    out = []
    vs = max(params["mach"] * params["cs"], 1e-3 * params["cs"])
    for l in range(sim.n_levels):
        for f in range(5):
            a, b = sim.get_field(l, f), orc.get_field(l, f)
            out.append((l, f, float(np.abs(a - b).max()) / (1.0 if f < 2 else vs)))
    return out


def force_sums(sim, orc, params):
    """(sum_c |w_c|, sum_c |w_c (rho_c - rho0)|, N) over the uncovered active cells of
    every level (the unfolded domain's, across mirror planes), with the oracle's
    densities"""
    GM, eps, rho0 = params["GM"], params["eps"], params["rho0"]
    tot = terms = 0.0
    cells = 0
    n = np.array(sim.n)
    n0 = np.array(sim.n0)
    mult = 1.0
    for d in range(3):  # a mirror plane doubles the sum (the unfolded domain's force)
        if sim.lo[d] == 0.0 and params["bc"][2 * d] == I.BC_REFLECT:
            mult *= 2.0
    for l in range(sim.n_levels):
        nl = n0 if l == 0 else n
        scale = (n / n0) / 2**l if l > 0 else np.ones(3)
        lo = np.array(sim.lo) * scale
        dx = (np.array(sim.hi) - np.array(sim.lo)) * scale / nl
        ax = [lo[d] + (np.arange(nl[d]) + 0.5) * dx[d] for d in range(3)]
        z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        r2 = x**2 + y**2 + z**2 + eps**2
        w = GM * np.prod(dx) * np.sqrt(x**2 + y**2 + z**2) / r2**1.5
        if l + 1 < sim.n_levels:
            lo_c = np.array(sim.lo) * (n / n0) / 2 ** (l + 1)
            q = np.rint((lo_c - lo) / dx).astype(int)
            w[q[2]:q[2] + n[2] // 2, q[1]:q[1] + n[1] // 2, q[0]:q[0] + n[0] // 2] = 0
        tot += w.sum()
        terms += (w * np.abs(orc.get_field(l, 0) - rho0)).sum()
        cells += int(np.count_nonzero(w))
    return mult * tot, mult * terms, cells


def force_bound(sim, orc, params, rho_err):
    """the bound of the module docstring for a measured density difference rho_err"""
    e = np.finfo(float).eps
    scale, terms, cells = force_sums(sim, orc, params)
    return (rho_err + 2 * e) * scale + cells * e * terms


def assert_parity(sim, orc, params, tol=TOL, label=""):
    errs = field_errors(sim, orc, params)
    worst = max(errs, key=lambda x: x[2])
    assert worst[2] <= tol, f"level {worst[0]} field {worst[1]}: {worst[2]:.3e}"
    rho_err = max(e for l, f, e in errs if f == 0)
    F, _ = sim.force()
    Fo = orc.force()
    bound = force_bound(sim, orc, params, rho_err)
    dF = np.abs(F - Fo).max()
    print(f"{label} fields {worst[2]:.2e} (rho {rho_err:.2e}); force {dF:.2e} abs, "
          f"{dF / max(np.abs(Fo).max(), 1e-300):.2e} rel, bound {bound:.2e}")
    assert dF <= bound, (F, Fo, bound)
    t, dt, bad = sim.status()
    assert bad == 0
    assert abs(t - orc.t) <= 1e-13 * max(orc.t, 1e-300)


def perturb_both(sim, orc, seed, amp=1e-2):
    """the same perturbed state in both: the library's FP64 state keeps 47 significant
    bits of a value written in, so the oracle starts from the values the library
    stored (read back exactly)"""
    n = sim.n
    for l in range(sim.n_levels):
        for f in range(5):
            base = orc.get_field(l, f)
            pert = I.smooth_perturbation(n[::-1], seed + 17 * l + f, amp)
            val = base * (1 + pert) if f < 2 else base + pert
            sim.set_field(l, f, val)
            orc.set_field(l, f, sim.get_field(l, f))
    for l in range(sim.n_levels - 1):
        orc.commup(l)
        sim.prolong(l)


@pytest.mark.parametrize("transport", TRANSPORTS, ids=TRANSPORT_IDS)
def test_uniform_flow_bitwise(transport):
    p = I.base_params(GM=0.0, L=0.0, chi=1.0, mach=0.7, flow_dir=(-0.6, 0.0, 0.8))
    sim, orc = pair(3, 24, 6.0, p, transport=transport)
    init = [[orc.get_field(l, f) for f in range(5)] for l in range(3)]
    sim.step(10)
    for l in range(3):
        for f in range(5):
            assert np.array_equal(sim.get_field(l, f), init[l][f]), (l, f)


def test_single_mesh_100_steps():
    """32^3 single mesh, Mach 0.5 wind, GM=0.01, softening 2 cells, chi=1: 100 steps."""
    cfg = I.single_mesh()
    p = cfg["params"]
    sim, orc = pair(1, cfg["n"], cfg["hi"][0], p)
    sim.step(100)
    orc.step(100)
    assert_parity(sim, orc, p)
    assert abs(sim.force()[0][0]) > 0


@pytest.mark.parametrize("transport", TRANSPORTS, ids=TRANSPORT_IDS)
def test_nested_100_coarse_steps(transport):
    """3 nested levels (ratio 2) of 32^3 with a Gaussian luminosity: 100 coarse steps."""
    p = I.base_params(GM=0.01, eps=0.125, chi=1.0, L=I.critical_luminosity(0.01, 1, 1, 5 / 3),
                      lum_sigma=0.125, mach=0.5)
    sim, orc = pair(3, 32, 8.0, p, transport=transport)
    sim.step(100)
    orc.step(100)
    assert_parity(sim, orc, p)


@pytest.mark.parametrize("bc", [
    (I.BC_PERIODIC,) * 6,
    (I.BC_REFLECT, I.BC_OUTFLOW, I.BC_REFLECT, I.BC_INFLOW, I.BC_OUTFLOW, I.BC_REFLECT),
    I.wind_bcs((0.0, 0.6, -0.8)),
])
@pytest.mark.parametrize("transport", TRANSPORTS, ids=TRANSPORT_IDS)
def test_perturbed_nested_boundaries(bc, transport):
    p = I.base_params(GM=0.02, eps=0.3, chi=0.4, L=0.03, lum_sigma=0.0, mach=0.8,
                      flow_dir=(0.0, 0.6, -0.8), bc=bc)
    sim, orc = pair(2, (24, 28, 32), (6.0, 7.0, 8.0), p, transport=transport)
    perturb_both(sim, orc, seed=3)
    sim.step(12)
    orc.step(12)
    assert_parity(sim, orc, p)


@pytest.mark.parametrize("transport", TRANSPORTS, ids=TRANSPORT_IDS)
def test_margin_boxes_equal_full_boxes(transport):
    """The active cells do not depend on the ghost margin the kernels sweep."""
    p = I.base_params(GM=0.01, eps=0.125, chi=1.0, L=0.05, lum_sigma=0.125, mach=0.9)
    a = binding.Sim(3, 24, (-6.0,) * 3, (6.0,) * 3, I.DEFAULT_G, p)
    b = binding.Sim(3, 24, (-6.0,) * 3, (6.0,) * 3, I.DEFAULT_G, p)
    a.set_transport(transport)
    b.set_transport(transport)
    b.debug_full_boxes(True)
    for s in (a, b):
        for l in range(3):
            for f in range(5):
                base = s.get_field(l, f)
                s.set_field(l, f, base + I.smooth_perturbation((24,) * 3, 40 + 5 * l + f, 5e-3))
        for l in range(2):
            s.prolong(l)
    a.step(15)
    b.step(15)
    for l in range(3):
        for f in range(5):
            assert np.array_equal(a.get_field(l, f), b.get_field(l, f)), (l, f)
    assert np.array_equal(a.force()[0], b.force()[0])


@pytest.mark.parametrize("precision", [binding.DF_FP64, binding.DF_FP32_STATE])
def test_tile_shapes_bitwise_equal(precision):
    """Tile shapes change only the order in which blocks visit a box: every shape gives
    the flat enumeration's result bit for bit, and autotuning does not advance the run."""
    p = I.base_params(GM=0.01, eps=0.125, chi=1.0, L=0.05, lum_sigma=0.125, mach=0.9)
    sims = []
    for shape in range(5):
        s = binding.Sim(3, 24, (-6.0,) * 3, (6.0,) * 3, I.DEFAULT_G, p, precision=precision)
        for l in range(3):
            for f in range(5):
                base = s.get_field(l, f)
                s.set_field(l, f, base + I.smooth_perturbation((24,) * 3, 70 + 5 * l + f, 5e-3))
        s.set_tile_shapes(shape)
        sims.append(s)
    tuned = sims[0]
    tuned.step(2)
    before = [tuned.get_field(l, f) for l in range(3) for f in range(5)]
    t0 = tuned.status()[0]
    shapes = tuned.autotune()
    assert all(0 <= v < 5 for row in shapes for v in row)
    assert tuned.status()[0] == t0
    assert all(np.array_equal(a, tuned.get_field(l, f))
               for (l, f), a in zip([(l, f) for l in range(3) for f in range(5)], before))
    tuned.step(8)
    for s in sims[1:]:
        s.step(10)
    for s in sims[1:]:
        for l in range(3):
            for f in range(5):
                assert np.array_equal(tuned.get_field(l, f), s.get_field(l, f)), (l, f)
        assert np.array_equal(tuned.force()[0], s.force()[0])


def test_fused_and_separate_transport_agree_fp32():
    """FP32 state: the fused sweeps and the separate kernels evaluate the same
    expressions; they differ only by the contraction of multiply-adds, so after 15
    coarse steps the fields agree to a few FP32 roundings of the perturbation."""
    p = I.base_params(GM=0.01, eps=0.125, chi=1.0, L=0.05, lum_sigma=0.125, mach=1.3,
                      flow_dir=(-0.6, 0.0, 0.8), bc=I.wind_bcs((-0.6, 0.0, 0.8)))
    sims = []
    for tr in TRANSPORTS:
        s = binding.Sim(3, (24, 28, 32), (-6.0, -7.0, -8.0), (6.0, 7.0, 8.0), I.DEFAULT_G, p,
                        precision=binding.DF_FP32_STATE)
        s.set_transport(tr)
        for l in range(3):
            for f in range(5):
                base = s.get_field(l, f)
                s.set_field(l, f, base + I.smooth_perturbation(base.shape, 90 + 5 * l + f, 5e-3))
        s.step(15)
        sims.append(s)
    a, b = sims
    vs = 1.3
    for l in range(3):
        for f in range(5):
            x, y = a.get_field(l, f), b.get_field(l, f)
            scale = 1.0 if f < 2 else vs
            assert np.abs(x - y).max() <= 2e-5 * scale, (l, f, np.abs(x - y).max())
    Fa, Fb = a.force()[0], b.force()[0]
    assert np.abs(Fa - Fb).max() <= 1e-4 * np.abs(Fb).max()


@pytest.mark.parametrize("transport", TRANSPORTS, ids=TRANSPORT_IDS)
def test_artificial_viscosity_parity(transport):
    """SubStep2 on: 3 nested levels with a strong compressive perturbation, the
    viscosity acting on every level; 10 coarse steps against the oracle."""
    p = I.base_params(GM=0.02, eps=0.3, chi=0.3, L=0.03, lum_sigma=0.3, mach=1.1, av_c2=2.0,
                      flow_dir=(0.0, 0.6, -0.8), bc=I.wind_bcs((0.0, 0.6, -0.8)))
    sim, orc = pair(3, 24, 6.0, p, transport=transport)
    perturb_both(sim, orc, seed=31, amp=0.15)
    sim.step(10)
    orc.step(10)
    assert_parity(sim, orc, p)


@pytest.mark.parametrize("precision", [binding.DF_FP64, binding.DF_FP32_STATE])
def test_sod_shock_tube_on_the_gpu(precision):
    """Sod's shock tube (t = 0.2, 200 cells, C2 = 2): FP64 equals the oracle to 1e-10;
    both precisions are within the oracle's L1 errors of the exact solution."""
    from test_oracle_sod import run_sod, sod_errors, sod_setup
    p, shape, lo, hi, fields, xc = sod_setup(2.0)
    sim = binding.Sim(1, shape, lo, hi, I.DEFAULT_G, p, precision=precision)
    for f in range(5):
        sim.set_field(0, f, fields[f])
    sim.step(250)
    t, _, bad = sim.status()
    assert bad == 0 and t == pytest.approx(0.2, rel=1e-12)
    er, ep, eu = sod_errors(lambda f: sim.get_field(0, f), t, xc)
    assert er < 0.005 and ep < 0.004 and eu < 0.009, (er, ep, eu)
    if precision == binding.DF_FP64:
        orc, _ = run_sod(2.0)
        for f in range(5):
            a, b = sim.get_field(0, f), orc.get_field(0, f)
            assert np.abs(a - b).max() <= TOL, (f, np.abs(a - b).max())


def test_inter_level_operators():
    """CommUp then CommMean on random states against the oracle (both from the values
    the library stored).  CommMean (level 0's band) sums in the stencils' arithmetic
    (double-float for the FP64 state) and stores the mean with 47 significant bits:
    within 2^-45 of the deviations from the background (up to ~1.5 here).  CommUp interpolates in the stencils' arithmetic, double-float for the
    FP64 state: each fine ghost is a coarse value plus a quarter of a limited slope,
    each within about 2^-45 of the deviations, so level 1 is held to 2^-43 of the
    largest value."""
    p = I.base_params()
    sim, orc = pair(2, 24, 6.0, p)
    rng = np.random.default_rng(9)
    shape = sim.full_shape()
    for l in range(2):
        for f in range(5):
            a = 1.0 + 0.1 * rng.standard_normal(shape)
            sim.set_full(l, f, a)
            orc.set_full(l, f, sim.get_full(l, f))
    sim.prolong(0)
    orc.commup(0)
    sim.restrict(0)
    orc.commmean(0)
    for l in range(2):
        for f in range(5):
            a, b = sim.get_full(l, f), orc.get_full(l, f)
            tol = 2.0**-45 if l == 0 else 2.0**-43
            assert np.abs(a - b).max() <= tol * np.abs(b).max(), (l, f)


def test_bc_fill_matches():
    p = I.base_params(bc=(I.BC_REFLECT, I.BC_PERIODIC, I.BC_INFLOW, I.BC_OUTFLOW, I.BC_OUTFLOW,
                          I.BC_REFLECT))
    p2 = dict(p, bc=(I.BC_PERIODIC,) * 2 + (I.BC_INFLOW, I.BC_OUTFLOW, I.BC_OUTFLOW, I.BC_REFLECT))
    sim, orc = pair(1, 16, 4.0, p2)
    rng = np.random.default_rng(2)
    for f in range(5):
        a = 1.0 + 0.1 * rng.standard_normal(sim.full_shape())
        sim.set_full(0, f, a)
        orc.set_full(0, f, sim.get_full(0, f))
    sim.fill_bc()
    orc.fill_bc()
    for f in range(5):
        # the library stores deviations from the background: full values are exact
        # up to the rounding of background + deviation
        a, b = sim.get_full(0, f), orc.get_full(0, f)
        assert np.abs(a - b).max() <= 4e-16 * np.abs(b).max(), f


def test_time_step_matches():
    """Eq. 55 limits per level and the step.  The FP64 state's per-cell sound speed
    and |v| are double-float (each within about 2^-44; the maxima, the minimum over
    levels and dt itself are FP64), so the limits are held to 2^-43."""
    p = I.base_params(GM=0.05, eps=0.3, chi=0.02, mach=1.5)
    sim, orc = pair(3, 24, 6.0, p)
    perturb_both(sim, orc, seed=8, amp=5e-2)
    dt, lv = sim.compute_dt()
    dto, lvo = orc.compute_dt()
    print(f"dt {abs(dt - dto) / dto:.2e} rel, limits {np.abs(lv / lvo - 1).max():.2e} rel")
    assert abs(dt - dto) <= 2.0**-43 * dto
    assert np.allclose(lv, lvo, rtol=2.0**-43, atol=0)


@pytest.mark.parametrize("transport", TRANSPORTS, ids=TRANSPORT_IDS)
def test_xi_search_mode_parity(transport):
    """Eq. 55-56 search each coarse step on the device (advective limit dominant:
    chi small, so the search drops sub-cycles), replayed from the CUDA graph."""
    from oracle import xi_search
    p = I.base_params(GM=0.02, eps=0.3, chi=0.005, mach=1.2, xi_mode=1)
    sim, orc = pair(3, 24, 6.0, p, transport=transport)
    perturb_both(sim, orc, seed=12, amp=2e-2)
    # a fast stream in a corner of level 0, away from the finer levels: the coarse
    # Courant limit binds, so the search drops second sub-cycles
    ax = -6.0 + (np.arange(24) + 0.5) * 0.5
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    bump = 3.0 * np.exp(-((x + 4.5) ** 2 + (y + 4.5) ** 2 + (z + 4.5) ** 2) / 0.5)
    for s_ in (sim, orc):
        s_.set_field(0, 2, s_.get_field(0, 2) - bump)
    dt, lim = sim.compute_dt()
    _, word = xi_search(lim, [24.0**3] * 3)
    assert 1 in word, word  # the case exercises dropped second sub-cycles
    sim.step(6)
    orc.step(6)
    assert_parity(sim, orc, p)


@pytest.mark.parametrize("precision", [binding.DF_FP64, binding.DF_FP32_STATE])
def test_xi_search_runs_in_pools(precision):
    """A run with the Eq. 55-56 search gives the same result in a pool, alone or
    mixed with fixed-sub-cycling runs, and agrees with a context."""
    p = I.base_params(GM=0.02, eps=0.3, chi=0.005, mach=1.2, xi_mode=1)
    q = I.base_params(GM=0.01, eps=0.3, chi=0.5, mach=0.6)
    lo, hi = (-6.0,) * 3, (6.0,) * 3
    ax = -6.0 + (np.arange(24) + 0.5) * 0.5
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    bump = 3.0 * np.exp(-((x + 4.5) ** 2 + (y + 4.5) ** 2 + (z + 4.5) ** 2) / 0.5)
    alone = binding.Pool(1 << 33, precision=precision)
    mix = binding.Pool(1 << 34, precision=precision)
    a = alone.admit(3, 24, lo, hi, I.DEFAULT_G, p)
    mix.admit(2, 32, lo, hi, I.DEFAULT_G, q)
    m = mix.admit(3, 24, lo, hi, I.DEFAULT_G, p)
    mix.admit(3, 24, lo, hi, I.DEFAULT_G, q)
    sim = binding.Sim(3, 24, lo, hi, I.DEFAULT_G, p, precision=precision)
    # the corner stream of test_xi_search_mode_parity: the search drops sub-cycles
    v0 = sim.get_field(0, 2) - bump
    sim.set_field(0, 2, v0)
    alone.set_field(a, 0, 2, v0)
    mix.set_field(m, 0, 2, v0)
    alone.step(5)
    mix.step(5)
    for l in range(3):
        for f in range(5):
            assert np.array_equal(alone.get_field(a, l, f), mix.get_field(m, l, f)), (l, f)
    qa, qm = alone.query()[a], mix.query()[m]
    assert np.array_equal(qa, qm)
    sim.step(5)
    tol = 1e-10 if precision == binding.DF_FP64 else 1e-5
    t, _, _ = sim.status()
    assert abs(t - qa[3]) <= 1e-12 * t
    for f in range(5):
        x, y = sim.get_field(2, f), alone.get_field(a, 2, f)
        assert np.abs(x - y).max() <= tol * (1.0 if f < 2 else 1.2), f


@pytest.mark.parametrize("transport", TRANSPORTS, ids=TRANSPORT_IDS)
def test_full_size_nested_config(transport):
    """The nested configuration at full size (3 levels of 64^3, coarse box [-8,8]^3,
    Mach 0.5, chi=1, Gaussian luminosity L_c) for 100 coarse steps, in the launch
    configuration the bench times (the oracle's OpenMP build, bitwise the plain one,
    keeps this to tens of seconds)."""
    cfg = I.nested()
    p = cfg["params"]
    lo, hi = cfg["lo"], cfg["hi"]
    sim = binding.Sim(cfg["n_levels"], cfg["n"], lo, hi, cfg["G"], p)
    sim.set_transport(transport)
    orc = Oracle(cfg["n_levels"], cfg["n"], lo, hi, cfg["G"], p, omp=True)
    sim.step(100)
    orc.step(100)
    assert_parity(sim, orc, p, label="nested 3x64^3, 100 coarse steps")
    F, _ = sim.force()
    assert np.abs(F[1:]).max() <= 1e-12 * abs(F[0]), F  # the transverse symmetry


def test_full_size_precision_config():
    """The precision configuration the bench's headline line times, at full size (5
    levels of 128^3, coarse box [-16,16]^3, Mach 1.2, chi=1, Gaussian luminosity L_c),
    FP64 state, the default transport form and tile order, 3 coarse steps (93 level
    steps) against the oracle's OpenMP build, every field of every level compared."""
    cfg = I.precision()
    p = cfg["params"]
    lo, hi = cfg["lo"], cfg["hi"]
    sim = binding.Sim(cfg["n_levels"], cfg["n"], lo, hi, cfg["G"], p)
    orc = Oracle(cfg["n_levels"], cfg["n"], lo, hi, cfg["G"], p, omp=True)
    sim.step(3)
    orc.step(3)
    assert_parity(sim, orc, p, label="precision 5x128^3, 3 coarse steps")
    F, _ = sim.force()
    assert np.abs(F[1:]).max() <= 1e-12 * abs(F[0]), F  # the transverse symmetry


def test_unhealthy_state_reported():
    p = I.base_params(GM=0.0, chi=0.5)
    sim = binding.Sim(1, 16, (-2.0,) * 3, (2.0,) * 3, I.DEFAULT_G, p)
    rho = sim.get_field(0, 0)
    rho[3, 4, 5] = -1.0
    sim.set_field(0, 0, rho)
    sim.step(1)
    with pytest.raises(binding.DfError) as ei:
        sim.force()
    assert ei.value.code == binding.DF_EUNHEALTHY


def test_checkpoint_resume_bitwise():
    p = I.base_params(GM=0.01, eps=0.125, chi=1.0, L=0.05, lum_sigma=0.125, mach=0.5)
    a = binding.Sim(3, 24, (-6.0,) * 3, (6.0,) * 3, I.DEFAULT_G, p)
    a.step(4)
    st, t = a.get_state()
    a.step(5)
    b = binding.Sim(3, 24, (-6.0,) * 3, (6.0,) * 3, I.DEFAULT_G, p)
    b.set_state(st, t)
    b.step(5)
    s1, t1 = a.get_state()
    s2, t2 = b.get_state()
    assert t1 == t2
    assert np.array_equal(s1, s2)


def test_fp32_state_close_to_fp64():
    """FP32 state with FP64 reductions: after 60 coarse steps the fields stay within
    1e-4 of the FP64 run (FP32 rounding accumulated over ~400 level steps) and the
    force within 1e-3 relative (the precision form's target)."""
    cfg = I.nested(n=32, n_levels=3, half=8.0, mach=1.2)
    p = cfg["params"]
    lo, hi = cfg["lo"], cfg["hi"]
    s64 = binding.Sim(3, 32, lo, hi, I.DEFAULT_G, p, precision=binding.DF_FP64)
    s32 = binding.Sim(3, 32, lo, hi, I.DEFAULT_G, p, precision=binding.DF_FP32_STATE)
    s64.step(60)
    s32.step(60)
    for l in range(3):
        for f in range(2):
            a, b = s32.get_field(l, f), s64.get_field(l, f)
            assert np.abs(a - b).max() < 1e-4, (l, f)
    F64 = s64.force()[0]
    F32 = s32.force()[0]
    assert np.abs(F32 - F64).max() <= 1e-3 * np.abs(F64).max(), (F32, F64)


def test_hot_path_division_within_one_ulp():
    """The FP64 division of the stencil kernels (Newton-Raphson on the hardware
    reciprocal estimate) against IEEE division, over the operand ranges it meets:
    densities near 1, 1 + a, and sums of same-signed slopes over many decades."""
    rng = np.random.default_rng(17)
    n = 1 << 20
    b = np.concatenate([1.0 + 0.3 * rng.standard_normal(n // 2),
                        np.exp(rng.uniform(-300, 300, n // 2)) * rng.choice([-1, 1], n // 2)])
    a = rng.standard_normal(n) * np.exp(rng.uniform(-30, 30, n))
    assert binding.check_division(a, b) <= 1.0


def test_adiabatic_subsonic_drag_on_the_gpu():
    """The GPU path at twice the oracle pin's resolution: 4 levels of 64^3 on
    [-16,16]^3, chi = 0, Mach 0.5: the drag settles near the linear-theory value
    -F0 I / M^2 (Ostriker 1999, the paper's Eq. 54 with F0 of Eq. 50)."""
    import math
    M, GM, nl, n, half = 0.5, 0.01, 4, 64, 16.0
    dxf = 2 * half / n / 2 ** (nl - 1)
    p = I.base_params(mach=M, GM=GM, chi=0.0, L=0.0, eps=2 * dxf)
    sim = binding.Sim(nl, n, (-half,) * 3, (half,) * 3, I.DEFAULT_G, p)
    Fth = -4 * math.pi * GM**2 * (0.5 * math.log((1 + M) / (1 - M)) - M) / M**2
    ratios = []
    while sim.t < 7.0:
        sim.step(4)
        F, along = sim.force()
        assert abs(along - F[0]) < 1e-18
        ratios.append((sim.t, along / Fth))
    late = [r for t, r in ratios if 3.5 < t < 7.0]
    assert late and all(0.95 < r < 1.06 for r in late), ratios
