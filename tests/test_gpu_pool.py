"""Batched runs (df_pool): uneven hierarchies stepped together by the work-list
kernels give, run by run, exactly what each run gives alone in its own context."""
import numpy as np
import pytest

from paper_1812_03191_gb300 import binding
from paper_1812_03191_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1812_03191_gb300 import build as B
    B.build()
    binding.load()


RUNS = [
    # (levels, n, half-box, params)
    (2, 24, 6.0, dict(mach=0.4, chi=0.7, L=0.0, GM=0.01, eps=0.25)),
    (3, 24, 6.0, dict(mach=1.3, chi=0.3, L=0.05, lum_sigma=0.2, GM=0.01, eps=0.2)),
    (1, 32, 4.0, dict(mach=0.8, chi=1.5, L=0.02, GM=0.02, eps=0.5)),
    (3, 32, 8.0, dict(mach=0.2, chi=2.0, L=0.0, GM=0.01, eps=0.125)),
]


@pytest.mark.parametrize("precision", [binding.DF_FP64, binding.DF_FP32_STATE])
def test_pool_mix_equals_runs_alone(precision):
    """Each run gives bitwise the same fields, force and time alone in a pool as in a
    mix of uneven runs (every pool launch uses the same work-list kernel, and every
    reduction has a fixed per-run order), and agrees with a standalone context
    within the parity tolerance (that path passes one work item by value, so the
    compiler may contract multiply-adds differently: rounding only)."""
    mix = binding.Pool(1 << 36, precision=precision)
    slots, alone, ctx = [], [], []
    for nl, n, half, over in RUNS:
        p = I.base_params(**over)
        lo, hi = (-half,) * 3, (half,) * 3
        slots.append(mix.admit(nl, n, lo, hi, I.DEFAULT_G, p))
        one = binding.Pool(1 << 34, precision=precision)
        one.admit(nl, n, lo, hi, I.DEFAULT_G, p)
        alone.append(one)
        ctx.append(binding.Sim(nl, n, lo, hi, I.DEFAULT_G, p, precision=precision))
    mix.step(7)
    for a, c in zip(alone, ctx):
        a.step(7)
        c.step(7)
    qm = mix.query()
    tol = 1e-10 if precision == binding.DF_FP64 else 1e-6
    for k, slot in enumerate(slots):
        qa = alone[k].query()
        assert np.array_equal(qm[slot], qa[0]), k
        p = I.base_params(**RUNS[k][3])
        vs = max(p["mach"] * p["cs"], 1e-3)
        for l in range(RUNS[k][0]):
            for f in range(5):
                a = mix.get_field(slot, l, f)
                assert np.array_equal(a, alone[k].get_field(0, l, f)), (k, l, f)
                b = ctx[k].get_field(l, f)
                assert np.abs(a - b).max() <= tol * (1.0 if f < 2 else vs), (k, l, f)
        F, _ = ctx[k].force()
        assert np.abs(qm[slot, :3] - F).max() <= 1e-6 * np.abs(F).max() + 1e-18
    # one launch carries the same op for every run that has it next: far fewer
    # launches than stepping the runs one by one
    assert mix.info()["launches"] < sum(a.info()["launches"] for a in alone)


class _View:
    def __init__(self, nl, n, half):
        self.n_levels, self.n, self.n0 = nl, (n,) * 3, (n,) * 3
        self.lo, self.hi = (-half,) * 3, (half,) * 3


def test_pool_runs_match_their_own_oracles():
    """Uneven FP64 runs stepped together by the batched work-list kernels: each run
    against its own oracle (fields to 1e-10, the force within the bound the density
    difference implies, the same time); then the same runs in FP32 state against
    the FP64 oracle, whose error is printed and bounded by the precision form's
    targets (force 1e-3 relative)."""
    from oracle import Oracle
    from test_gpu_parity import force_bound
    for precision in (binding.DF_FP64, binding.DF_FP32_STATE):
        pool = binding.Pool(1 << 36, precision=precision)
        slots, orcs = [], []
        for nl, n, half, over in RUNS:
            p = I.base_params(**over)
            slots.append(pool.admit(nl, n, (-half,) * 3, (half,) * 3, I.DEFAULT_G, p))
            orcs.append(Oracle(nl, n, (-half,) * 3, (half,) * 3, I.DEFAULT_G, p))
        pool.step(8)
        for k, ((nl, n, half, over), slot, orc) in enumerate(zip(RUNS, slots, orcs)):
            orc.step(8)
            p = I.base_params(**over)
            vs = max(p["mach"] * p["cs"], 1e-3)
            worst = rho_err = 0.0
            for l in range(nl):
                for f in range(5):
                    e = np.abs(pool.get_field(slot, l, f) - orc.get_field(l, f)).max()
                    e /= 1.0 if f < 2 else vs
                    worst = max(worst, e)
                    rho_err = max(rho_err, e) if f == 0 else rho_err
            F, t = pool.force(slot)
            Fo = orc.force()
            dF = np.abs(F - Fo).max()
            print(f"precision {precision} run {k}: fields {worst:.2e}, force {dF:.2e} abs, "
                  f"{dF / np.abs(Fo).max():.2e} rel")
            if precision == binding.DF_FP64:
                assert worst <= 1e-10, (k, worst)
                assert dF <= force_bound(_View(nl, n, half), orc, p, rho_err), (k, F, Fo)
                assert abs(t - orc.t) <= 1e-13 * orc.t
            else:
                assert worst <= 1e-4, (k, worst)
                assert dF <= 1e-3 * np.abs(Fo).max(), (k, F, Fo)
            orc.close()
        pool.close()


def test_pool_budget_admission_and_release():
    shape = (2, 24)
    need = binding.run_bytes(shape[0], shape[1], I.DEFAULT_G)
    pool = binding.Pool(2 * need + need // 2)
    p = I.base_params()
    lo, hi = (-6.0,) * 3, (6.0,) * 3
    a = pool.admit(*shape, lo, hi, I.DEFAULT_G, p)
    b = pool.admit(*shape, lo, hi, I.DEFAULT_G, p)
    assert a is not None and b is not None
    assert pool.admit(*shape, lo, hi, I.DEFAULT_G, p) is None  # over budget
    assert pool.info()["active"] == 2
    pool.release(a)
    c = pool.admit(*shape, lo, hi, I.DEFAULT_G, p)
    assert c == a  # the freed slot is reused
    pool.step(2)
    assert np.isfinite(pool.query()[[b, c], :3]).all()


def test_autotune_keeps_state_and_results():
    p = I.base_params(mach=0.9, chi=0.5, L=0.03, lum_sigma=0.3)
    lo, hi = (-6.0,) * 3, (6.0,) * 3
    pa, pb = binding.Pool(1 << 34), binding.Pool(1 << 34)
    for pool in (pa, pb):
        pool.admit(3, 24, lo, hi, I.DEFAULT_G, p)
        pool.admit(2, 32, lo, hi, I.DEFAULT_G, dict(p, mach=1.4))
        pool.step(2)
    tiles = pb.autotune()
    assert len(tiles) == binding.POOL_OPS and all(1 <= t <= 32 for t in tiles)
    pa.set_tile_shapes(3)  # a fixed tile shape on one side, the tuned ones on the other
    pa.step(3)
    pb.step(3)
    for slot in (0, 1):
        for f in range(5):
            assert np.array_equal(pa.get_field(slot, 0, f), pb.get_field(slot, 0, f))
    assert np.array_equal(pa.query(), pb.query())
