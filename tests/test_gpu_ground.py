"""A ground level with its own cell count (df_create_ground; the hierarchy of
Sec. 4.1.1 whose first level covers a quarter of the ground) on the GPU: parity with
the oracle, the paper's low-Mach geometry (quadrant plus quarter first level), FP32
state against FP64, pools, checkpoints and the autotuner's state restore."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1812_03191_gb300 import binding
from paper_1812_03191_gb300 import inputs as I
from test_gpu_parity import TRANSPORTS, TRANSPORT_IDS, field_errors, force_bound

pytestmark = pytest.mark.gpu

HALF = 6.0
N = 24
N0 = 2 * N
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1812_03191_gb300 import build as B
    B.build()
    binding.load()


def _params(**over):
    p = I.base_params(GM=0.02, eps=0.3, chi=0.4, L=0.03, lum_sigma=0.0, mach=0.8,
                      flow_dir=(0.0, 0.6, -0.8), bc=I.wind_bcs((0.0, 0.6, -0.8)))
    p.update(over)
    return p


def _perturb(runs, seed, amp=1e-2):
    """the same smooth perturbation on every level of every run (Sim or Oracle)"""
    for l in range(runs[0].n_levels):
        for f in range(5):
            base = runs[0].get_field(l, f)
            pert = I.smooth_perturbation(base.shape, seed + 17 * l + f, amp)
            val = base * (1 + pert) if f < 2 else base + pert
            # the first run's stored values (its FP64 state keeps 47 significant bits)
            runs[0].set_field(l, f, val)
            val = runs[0].get_field(l, f)
            for r in runs[1:]:
                r.set_field(l, f, val)
    for l in range(runs[0].n_levels - 1):
        for r in runs:
            r.commup(l) if isinstance(r, Oracle) else r.prolong(l)


def _assert_parity(sim, orc, p, steps):
    sim.step(steps)
    orc.step(steps)
    errs = field_errors(sim, orc, p)
    worst = max(errs, key=lambda e: e[2])
    assert worst[2] <= TOL, worst
    F, Fo = sim.force()[0], orc.force()
    bound = force_bound(sim, orc, p, max(e for l, f, e in errs if f == 0))
    dF = np.abs(F - Fo).max()
    print(f"ground: fields {worst[2]:.2e}; force {dF:.2e} abs, "
          f"{dF / np.abs(Fo).max():.2e} rel, bound {bound:.2e}")
    assert dF <= bound, (F, Fo, bound)
    assert sim.status()[2] == 0


@pytest.mark.parametrize("transport", TRANSPORTS, ids=TRANSPORT_IDS)
def test_ground_level_parity_with_the_oracle(transport):
    p = _params()
    lo, hi = (-HALF,) * 3, (HALF,) * 3
    sim = binding.Sim(3, N, lo, hi, I.DEFAULT_G, p, n0=N0)
    sim.set_transport(transport)
    orc = Oracle(3, N, lo, hi, I.DEFAULT_G, p, n0=N0)
    _perturb([sim, orc], seed=31)
    _assert_parity(sim, orc, p, 10)


@pytest.mark.parametrize("transport", TRANSPORTS, ids=TRANSPORT_IDS)
def test_low_mach_geometry_of_the_paper_parity(transport):
    """quadrant domain, ground of n x n x 2n cells, levels of n/2 x n/2 x n, the
    first over a quarter of the ground, Eq. 55-56 search on"""
    cfg = I.quadrant(n=24, n_levels=3, half=HALF, mach=0.3, quarter=True, GM=0.05, chi=0.3,
                     L=0.02, xi_mode=1)
    p = cfg["params"]
    sim = binding.Sim(3, cfg["n"], cfg["lo"], cfg["hi"], cfg["G"], p, n0=cfg["n0"])
    sim.set_transport(transport)
    orc = Oracle(3, cfg["n"], cfg["lo"], cfg["hi"], cfg["G"], p, n0=cfg["n0"])
    _assert_parity(sim, orc, p, 12)
    F = sim.force()[0]
    assert F[0] == 0.0 and F[1] == 0.0 and abs(F[2]) > 0


def test_fp32_ground_level_close_to_fp64():
    cfg = I.quadrant(n=32, n_levels=4, half=8.0, mach=1.2, quarter=True, GM=0.01, chi=0.5,
                     L=0.02)
    runs = [binding.Sim(cfg["n_levels"], cfg["n"], cfg["lo"], cfg["hi"], cfg["G"],
                        cfg["params"], precision=pr, n0=cfg["n0"])
            for pr in (binding.DF_FP64, binding.DF_FP32_STATE)]
    for r in runs:
        r.step(40)
    for l in range(cfg["n_levels"]):
        for f in range(2):
            a, b = runs[1].get_field(l, f), runs[0].get_field(l, f)
            assert np.abs(a - b).max() < 1e-4, (l, f)
    F64, F32 = runs[0].force()[0], runs[1].force()[0]
    assert np.abs(F32 - F64).max() <= 1e-3 * np.abs(F64).max(), (F32, F64)


def test_ground_runs_share_a_pool():
    """ground-level runs next to a plain one in one pool: each gets the bits of a
    pool of its own, and the HBM accounting follows df_run_bytes_ground"""
    lo, hi = (-HALF,) * 3, (HALF,) * 3
    cases = [(3, N0), (2, N), (3, N0 + 8)]
    mix = binding.Pool(8 << 30, precision=binding.DF_FP32_STATE)
    runs = []
    for nl, n0 in cases:
        p = _params(mach=1.1)
        alone = binding.Pool(4 << 30, precision=binding.DF_FP32_STATE)
        runs.append((nl, n0, mix.admit(nl, N, lo, hi, I.DEFAULT_G, p, n0=n0), alone,
                     alone.admit(nl, N, lo, hi, I.DEFAULT_G, p, n0=n0)))
    used = mix.info()["used"]
    assert used == sum(binding.run_bytes(nl, N, I.DEFAULT_G, binding.DF_FP32_STATE, n0=n0)
                       for nl, n0 in cases)
    mix.step(8)
    for nl, n0, m, alone, a in runs:
        alone.step(8)
        for l in range(nl):
            for f in range(5):
                assert np.array_equal(mix.get_field(m, l, f), alone.get_field(a, l, f)), (n0, l, f)
        alone.close()
    mix.close()


def test_checkpoint_resume_with_a_ground_level():
    p = _params()
    lo, hi = (-HALF,) * 3, (HALF,) * 3
    a = binding.Sim(3, N, lo, hi, I.DEFAULT_G, p, n0=N0)
    a.step(4)
    state, t = a.get_state()
    assert state.size == 3 * 5 * int(np.prod(a.full_shape(0)))
    a.step(5)
    b = binding.Sim(3, N, lo, hi, I.DEFAULT_G, p, n0=N0)
    b.set_state(state, t)
    b.step(5)
    for l in range(3):
        for f in range(5):
            assert np.array_equal(a.get_field(l, f), b.get_field(l, f)), (l, f)


def test_autotune_restores_a_ground_level_run():
    """the tuner steps the runs to time them and puts their state back: levels of
    different sizes come back bitwise"""
    p = _params()
    lo, hi = (-HALF,) * 3, (HALF,) * 3
    s = binding.Sim(3, N, lo, hi, I.DEFAULT_G, p, n0=N0, precision=binding.DF_FP32_STATE)
    s.step(3)
    before = [[s.get_field(l, f) for f in range(5)] for l in range(3)]
    s.autotune()
    for l in range(3):
        for f in range(5):
            assert np.array_equal(s.get_field(l, f), before[l][f]), (l, f)


def test_ground_level_geometry_is_checked():
    p = _params()
    lo, hi = (-HALF,) * 3, (HALF,) * 3
    with pytest.raises(binding.DfError):  # level 1 would not sit on ground faces
        binding.Sim(2, N, lo, (10.0, HALF, HALF), I.DEFAULT_G, p, n0=(56, N0, N0))
    with pytest.raises(binding.DfError):  # the ground is smaller than its child's stencil
        binding.Sim(2, N, lo, hi, I.DEFAULT_G, p, n0=N // 2 + 8)
