"""Mirror planes (the quadrant domain of Sec. 3.4) on the GPU: parity with the
oracle, the unfolded whole domain reproduced by the GPU itself, FP32 state against
FP64, and mirrored and unmirrored runs stepped together in one pool."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1812_03191_gb300 import binding
from paper_1812_03191_gb300 import inputs as I
from test_gpu_parity import TRANSPORTS, TRANSPORT_IDS, assert_parity, perturb_both

pytestmark = pytest.mark.gpu

HALF = 3.0
N = 24


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1812_03191_gb300 import build as B
    B.build()
    binding.load()


def _params(mirror, **over):
    bc = [I.BC_REFLECT] * 4 + [I.BC_INFLOW, I.BC_OUTFLOW]
    if not mirror[1]:
        bc[2] = bc[3] = I.BC_OUTFLOW
    p = I.base_params(gamma=1.4, mach=0.8, flow_dir=(0.0, 0.0, 1.0), GM=0.05, eps=0.0,
                      chi=0.3, L=0.02, lum_sigma=0.0, bc=tuple(bc))
    p.update(over)
    return p


def _geometry(mirror):
    n = tuple(N // 2 if m else N for m in mirror) + (N,)
    lo = tuple(0.0 if m else -HALF for m in mirror) + (-HALF,)
    return n, lo, (HALF,) * 3


CASES = [(1, {}), (2, {}), (3, dict(xi_mode=1)), (2, dict(lum_sigma=0.3, av_c2=1.0))]
CASE_IDS = ["1level", "2levels", "3levels_xi", "2levels_gauss_visc"]


@pytest.mark.parametrize("transport", TRANSPORTS, ids=TRANSPORT_IDS)
@pytest.mark.parametrize("n_levels,over", CASES, ids=CASE_IDS)
@pytest.mark.parametrize("mirror", [(True, True), (True, False)], ids=["quadrant", "half"])
def test_mirror_parity_with_the_oracle(mirror, n_levels, over, transport):
    p = _params(mirror, **over)
    n, lo, hi = _geometry(mirror)
    sim = binding.Sim(n_levels, n, lo, hi, I.DEFAULT_G, p, precision=binding.DF_FP64)
    sim.set_transport(transport)
    orc = Oracle(n_levels, n, lo, hi, I.DEFAULT_G, p)
    sim.step(12)
    orc.step(12)
    assert_parity(sim, orc, p)
    F, _ = sim.force()
    assert F[0] == 0.0 and (F[1] == 0.0) == mirror[1] and abs(F[2]) > 0


@pytest.mark.parametrize("transport", TRANSPORTS, ids=TRANSPORT_IDS)
def test_perturbed_quadrant_parity(transport):
    """an asymmetric perturbation of every level (the quadrant's own state need not
    be symmetric) with a supersonic wind"""
    p = _params((True, True), mach=1.5, GM=0.02, L=0.05)
    n, lo, hi = _geometry((True, True))
    sim = binding.Sim(3, n, lo, hi, I.DEFAULT_G, p, precision=binding.DF_FP64)
    sim.set_transport(transport)
    orc = Oracle(3, n, lo, hi, I.DEFAULT_G, p)
    perturb_both(sim, orc, seed=21)
    sim.step(10)
    orc.step(10)
    assert_parity(sim, orc, p)


@pytest.mark.parametrize("precision", [binding.DF_FP64, binding.DF_FP32_STATE])
def test_quadrant_reproduces_the_whole_domain_on_the_gpu(precision):
    """the GPU's quadrant run against the GPU's whole-domain run of the unfolded
    problem: same fields on x, y > 0 and the same force"""
    mirror = (True, True)
    p = _params(mirror)
    n, lo, hi = _geometry(mirror)
    part = binding.Sim(3, n, lo, hi, I.DEFAULT_G, p, precision=precision)
    full = binding.Sim(3, N, (-HALF,) * 3, (HALF,) * 3, I.DEFAULT_G, p, precision=precision)
    part.step(12)
    full.step(12)
    tol = 1e-12 if precision == binding.DF_FP64 else 2e-6
    for l in range(3):
        for f in range(5):
            a = full.get_field(l, f)[:, N // 2:, N // 2:]
            b = part.get_field(l, f)
            assert np.abs(a - b).max() <= tol * 2.0, (l, f, np.abs(a - b).max())
    Ff, Fp = full.force()[0], part.force()[0]
    assert abs(Fp[2] - Ff[2]) <= (1e-10 if precision == binding.DF_FP64 else 1e-4) * abs(Ff[2])
    assert abs(Ff[0]) <= 1e-6 * abs(Ff[2]) and abs(Ff[1]) <= 1e-6 * abs(Ff[2])


def test_fp32_quadrant_close_to_fp64():
    cfg = I.quadrant(n=32, n_levels=4, half=8.0, mach=1.2, GM=0.01, chi=0.5, L=0.02)
    runs = [binding.Sim(cfg["n_levels"], cfg["n"], cfg["lo"], cfg["hi"], cfg["G"],
                        cfg["params"], precision=pr)
            for pr in (binding.DF_FP64, binding.DF_FP32_STATE)]
    for r in runs:
        r.step(40)
    for l in range(cfg["n_levels"]):
        for f in range(2):
            a, b = runs[1].get_field(l, f), runs[0].get_field(l, f)
            assert np.abs(a - b).max() < 1e-4, (l, f)
    F64, F32 = runs[0].force()[0], runs[1].force()[0]
    assert np.abs(F32 - F64).max() <= 1e-3 * np.abs(F64).max(), (F32, F64)


def test_mirrored_and_whole_runs_share_a_pool():
    """a quadrant run, a half run and a whole-domain run admitted together: the
    merged launches give each run the bits it gets in a pool of its own, and a
    context agrees with the pool to FP32 rounding"""
    cases = [((True, True), 3), ((True, False), 2), ((False, False), 2)]
    mix = binding.Pool(4 << 30, precision=binding.DF_FP32_STATE)
    runs = []
    for mirror, nl in cases:
        p = _params(mirror)
        if mirror == (False, False):
            n, lo, hi = N, (-HALF,) * 3, (HALF,) * 3
        else:
            n, lo, hi = _geometry(mirror)
        alone = binding.Pool(2 << 30, precision=binding.DF_FP32_STATE)
        runs.append((mirror, nl, mix.admit(nl, n, lo, hi, I.DEFAULT_G, p), alone,
                     alone.admit(nl, n, lo, hi, I.DEFAULT_G, p),
                     binding.Sim(nl, n, lo, hi, I.DEFAULT_G, p, precision=binding.DF_FP32_STATE)))
    mix.step(10)
    for mirror, nl, m, alone, a, sim in runs:
        alone.step(10)
        sim.step(10)
        for l in range(nl):
            for f in range(5):
                x, y = mix.get_field(m, l, f), alone.get_field(a, l, f)
                assert np.array_equal(x, y), (mirror, l, f)
                z = sim.get_field(l, f)
                assert np.abs(x - z).max() <= 2e-5 * (1.0 if f < 2 else 0.8), (mirror, l, f)
        alone.close()
    mix.close()


def test_finer_levels_on_a_face_need_a_mirror():
    p = _params((True, True), bc=(I.BC_OUTFLOW,) + (I.BC_REFLECT,) * 3 + (I.BC_INFLOW,) * 2)
    n, lo, hi = _geometry((True, True))
    with pytest.raises(binding.DfError):
        binding.Sim(2, n, lo, hi, I.DEFAULT_G, p)
    binding.Sim(1, n, lo, hi, I.DEFAULT_G, p).close()
