"""Serving loop: stopping rule on the host (CPU) and continuous batching on the GPU,
where every request's result must be the same alone and in the mix."""
import numpy as np
import pytest

from paper_1812_03191_gb300 import binding
from paper_1812_03191_gb300 import inputs as I
from paper_1812_03191_gb300 import serve as S


def _spec(n_levels=2, n=24, half=6.0, **over):
    return dict(n_levels=n_levels, n=n, lo=(-half,) * 3, hi=(half,) * 3, G=I.DEFAULT_G,
                params=I.base_params(**over))


def test_crossing_time_and_direction():
    sp = _spec(n_levels=3, half=8.0, mach=0.5)
    # finest level half-width 8/4 = 2; t_cross = 2 * 2 / (cs + V)
    assert S.crossing_time(sp) == pytest.approx(4.0 / 1.5)
    # the wind blows along -x: the perturber moves along +x
    assert S.along_motion(np.array([2.0, 5.0, 7.0]), sp) == pytest.approx(2.0)


def test_convergence_rule():
    tr = S.Track(0, _spec(), 0.0, 0.0, t_cross=1.0)
    for k in range(30):
        t = 0.1 * k
        tr.ts.append(t)
        tr.Fs.append(1.0 - np.exp(-t))  # still moving early, settles later
    assert not tr.converged(1e-3)  # F(2.9) - F(1.9) is still ~10 % of F
    tr2 = S.Track(0, _spec(), 0.0, 0.0, t_cross=1.0)
    for k in range(40):
        tr2.ts.append(0.1 * k)
        tr2.Fs.append(3.0)
    assert tr2.converged(1e-3)
    tr3 = S.Track(0, _spec(), 0.0, 0.0, t_cross=1.0)
    for k in range(5):
        tr3.ts.append(0.1 * k)
        tr3.Fs.append(3.0)
    assert not tr3.converged(1e-3)  # before 2 t_cross


def test_batch_sizes_follow_the_stopping_rule():
    """The host reads the runs after a batch of coarse steps: long before 2 t_cross a
    batch covers the steps to it, near or past it `check_every` steps, never past the
    step cap, and a single step while requests wait for room."""
    srv = S.Server.__new__(S.Server)
    srv.step_cap, srv.check_every, srv.step_s, srv.max_slots = 100, 8, 1e-3, None
    early = S.Track(0, _spec(), 0.0, 0.0, t_cross=1.0)
    early.ts, early.steps = [0.0, 0.01], 2  # dt = 0.01: 198 steps to t = 2
    assert srv._batch({0: early}, False, None) == 98  # the step cap binds
    srv.step_cap = 1000
    assert srv._batch({0: early}, False, None) == 199
    late = S.Track(1, _spec(), 0.0, 0.0, t_cross=1.0)
    late.ts, late.steps = [2.5, 2.51], 300
    assert srv._batch({0: early, 1: late}, False, None) == 8
    assert srv._batch({0: early}, True, None) == 1  # a request waits for room
    # the next arrival in 50 ms at 1 ms per step
    assert srv._batch({0: early}, False, 0.05) == 51
    fresh = S.Track(2, _spec(), 0.0, 0.0, t_cross=1.0)  # no step yet: dt unknown
    assert srv._batch({2: fresh}, False, None) == 8
    # one slot only (the sequential baseline): a waiting request cannot be admitted
    # before the run finishes, so it does not shorten the batch
    srv.max_slots = 1
    assert srv._batch({0: early}, True, 0.01) == 199
    srv.max_slots = None


def test_oversize_request_rejected_alone():
    """A request that cannot fit even an empty pool gets an error result; the server
    neither raises nor stops (no GPU work: the pool object is a stand-in)."""

    class FakePool:
        def admit(self, *a, **k):
            return None

    srv = S.Server.__new__(S.Server)
    srv.pool, srv.budget, srv.precision = FakePool(), 1000, binding.DF_FP32_STATE
    srv.tiles, srv.max_active, srv.max_slots = None, 0, None
    orig = binding.run_bytes
    binding.run_bytes = lambda *a, **k: 10**9
    try:
        results, summary = srv.run([(0.0, _spec())], sleep=lambda s: None)
    finally:
        binding.run_bytes = orig
    assert len(results) == 1 and results[0].error and "budget" in results[0].error
    assert summary["failed"] == 1 and summary["requests"] == 1


@pytest.mark.gpu
def test_unhealthy_request_fails_alone():
    """A NaN planted in one run's density (on the host, through the pool API) retires
    that request with an error; every other request finishes with bitwise the result
    it has alone."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1812_03191_gb300 import build as B
    B.build()
    reqs = [(0.0, _spec(n_levels=2, n=24, mach=0.3 + 0.4 * k, chi=0.5, L=0.02, lum_sigma=0.3))
            for k in range(4)]
    bad = 2

    def plant(pool, slot, rid):
        if rid == bad:
            rho = pool.get_field(slot, 1, 0)
            rho[5, 6, 7] = np.nan
            pool.set_field(slot, 1, 0, rho)

    one = binding.run_bytes(2, 24, I.DEFAULT_G, binding.DF_FP32_STATE)
    srv = S.Server(8 * one, precision=binding.DF_FP32_STATE, tol=1e-12, step_cap=7)
    results, summary = srv.run(reqs, on_admit=plant)
    srv.close()
    assert summary["requests"] == 4 and summary["failed"] == 1
    for r in results:
        if r.rid == bad:
            assert r.error and "unhealthy" in r.error
            continue
        assert r.error is None and r.steps == 7
        sp = reqs[r.rid][1]
        alone = binding.Pool(one * 2, precision=binding.DF_FP32_STATE)
        alone.admit(sp["n_levels"], sp["n"], sp["lo"], sp["hi"], sp["G"], sp["params"])
        alone.step(r.steps)
        q = alone.query()[0]
        alone.close()
        assert np.array_equal(q[:3], r.F) and q[3] == r.t, r.rid


@pytest.mark.gpu
def test_requests_same_alone_and_in_the_mix():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1812_03191_gb300 import build as B
    B.build()
    rng = np.random.default_rng(4)
    reqs = []
    for k in range(7):
        nl = int(rng.choice([2, 3]))
        sp = _spec(n_levels=nl, n=24, mach=float(rng.uniform(0.2, 2.0)),
                   chi=float(rng.uniform(0.3, 2.0)), L=float(rng.choice([0.0, 0.05])),
                   lum_sigma=0.3)
        reqs.append((0.0, sp))
    # room for about three runs at once: later requests wait for freed slots
    one = binding.run_bytes(3, 24, I.DEFAULT_G, binding.DF_FP32_STATE)
    srv = S.Server(3 * one, precision=binding.DF_FP32_STATE, tol=1e-12, step_cap=9)
    results, summary = srv.run(reqs)
    srv.close()
    # all arrive at once; the budget holds three, the rest queue for freed slots
    assert summary["requests"] == len(reqs) and srv.max_active >= 2
    assert all(r.capped and r.steps == 9 for r in results)
    for r in results:
        sp = reqs[r.rid][1]
        alone = binding.Pool(one * 2, precision=binding.DF_FP32_STATE)
        alone.admit(sp["n_levels"], sp["n"], sp["lo"], sp["hi"], sp["G"], sp["params"])
        alone.step(r.steps)
        q = alone.query()[0]
        alone.close()
        assert np.array_equal(q[:3], r.F) and q[3] == r.t, r.rid
