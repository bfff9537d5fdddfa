"""The allocation-free force entry point agrees with the context's force reduction
and with the oracle.

df_force_level_noalloc serves callers that cannot call cudaMalloc: a process whose
device memory is fully reserved by another allocator, a loop that cannot take
cudaMalloc's implicit synchronisation, a sandboxed plug-in that may not allocate.
It keeps its scratch in a fixed device array shared by every call, so this test
checks two calls in a row, on different states, against df_force_now; the same on
a quadrant-domain context (mirror planes); a given density against the oracle's
force sum; and that oversize input and covered boxes outside the level are
rejected.  Collected last: it runs alone in a fresh process as well as after every
other test.
"""
import numpy as np
import pytest

from paper_1812_03191_gb300 import binding
from paper_1812_03191_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-10  # the force tolerance of the other GPU tests


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1812_03191_gb300 import build as B
    B.build()
    binding.load()


def _level_geometry(n, lo, hi, level):
    """active cells, lower corner and cell size of a level, and the box its child
    covers (offset, extent) in its active cells"""
    dx = [(hi[d] - lo[d]) / 2**level / n[d] for d in range(3)]
    lo_l = [lo[d] / 2**level for d in range(3)]
    off = [int(round(-lo[d] / (2 * (hi[d] - lo[d])) * n[d])) for d in range(3)]
    return lo_l, dx, off, [n[d] // 2 for d in range(3)]


def _noalloc_total(levels, n, G, lo, hi, params, stream, mirror=0):
    """sum over levels of the allocation-free per-level force; levels: the padded
    full density of each level (host arrays)"""
    import torch
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    total = np.zeros(3)
    for l, full in enumerate(levels):
        rho = torch.from_numpy(np.ascontiguousarray(full).ravel().copy()).cuda()
        lo_l, dx, off, ext = _level_geometry(n, lo, hi, l)
        child_off = child_n = None
        if l + 1 < len(levels):
            child_off, child_n = off, ext
        binding.force_level_noalloc(rho.data_ptr(), n, G, lo_l, dx, child_off, child_n,
                                    params["GM"], params["eps"], params["rho0"],
                                    out.data_ptr(), stream, mirror=mirror)
        torch.cuda.current_stream().synchronize()
        total += out.cpu().numpy()
    return total


@pytest.mark.parametrize("n_levels", [1, 3])
def test_noalloc_force_matches_context_force_twice(n_levels):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    half = 6.0
    lo, hi = (-half,) * 3, (half,) * 3
    p = I.base_params(GM=0.013, eps=0.2, chi=0.5, L=0.05, lum_sigma=0.25, mach=0.7)
    sim = binding.Sim(n_levels, 24, lo, hi, I.DEFAULT_G, p)
    for call in range(2):
        sim.step(3 + 4 * call)  # a different state for each call
        ref = sim.force_now()
        full = [sim.get_full(l, 0) for l in range(n_levels)]
        got = _noalloc_total(full, sim.n, sim.G, lo, hi, p, stream)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        print(f"levels {n_levels} call {call}: relative force difference {err:.2e}")
        assert err <= TOL, (call, got, ref)
        assert np.abs(ref).max() > 0
    sim.close()


def test_noalloc_force_on_a_quadrant_context():
    """Mirror planes x = 0 and y = 0 (Sec. 3.4 quadrant domain): with the mirror mask
    the per-level sums give the unfolded domain's force, as df_force_now does."""
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    cfg = I.quadrant(n=32, n_levels=3, half=8.0, mach=0.8, GM=0.02, eps=0.3, chi=0.5,
                     L=0.05, lum_sigma=0.3)
    sim = binding.Sim(cfg["n_levels"], cfg["n"], cfg["lo"], cfg["hi"], cfg["G"],
                      cfg["params"])
    for call in range(2):
        sim.step(4 + 3 * call)
        ref = sim.force_now()
        full = [sim.get_full(l, 0) for l in range(cfg["n_levels"])]
        got = _noalloc_total(full, sim.n, sim.G, cfg["lo"], cfg["hi"], cfg["params"], stream,
                             mirror=3)
        assert ref[0] == 0.0 and ref[1] == 0.0 and got[0] == 0.0 and got[1] == 0.0
        assert abs(got[2] - ref[2]) <= TOL * abs(ref[2]), (call, got, ref)
        assert ref[2] != 0.0
    sim.close()


def test_noalloc_force_matches_the_oracle_on_a_given_density():
    """The same density on both sides: the oracle's force sum (Eq. 18 level by level,
    covered cells excluded) and the allocation-free per-level sums agree."""
    import torch
    from oracle import Oracle
    stream = torch.cuda.current_stream().cuda_stream
    n, nl, half, G = 24, 3, 6.0, I.DEFAULT_G
    lo, hi = (-half,) * 3, (half,) * 3
    p = I.base_params(GM=0.011, eps=0.15)
    orc = Oracle(nl, n, lo, hi, G, p)
    rng = np.random.default_rng(7)
    for l in range(nl):
        orc.set_field(l, 0, 1.0 + 0.05 * rng.standard_normal((n, n, n)))
    ref = orc.force()
    full = [orc.get_full(l, 0) for l in range(nl)]
    for call in range(2):
        got = _noalloc_total(full, (n, n, n), G, lo, hi, p, stream)
        assert np.abs(got - ref).max() <= TOL * np.abs(ref).max(), (call, got, ref)
    orc.close()


def test_noalloc_rejects_more_cells_than_its_scratch():
    import torch
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    rho = torch.ones(8, dtype=torch.float64, device="cuda")
    n = (256, 256, 128)  # 8,388,608 active cells > DF_NOALLOC_MAX_CELLS
    with pytest.raises(binding.DfError) as ei:
        binding.force_level_noalloc(rho.data_ptr(), n, 0, (0, 0, 0), (1, 1, 1), None, None,
                                    1.0, 0.0, 1.0, out.data_ptr(), None)
    assert ei.value.code == binding.DF_EINVAL
    assert "exceed" in str(ei.value)


@pytest.mark.parametrize("off,ext,mirror", [((-1, 4, 4), (8, 8, 8), 0),
                                            ((4, 4, 4), (0, 8, 8), 0),
                                            ((4, 4, 12), (8, 8, 8), 0),
                                            ((4, 4, 4), (8, 8, 8), 8)])
def test_noalloc_rejects_a_covered_box_outside_the_level(off, ext, mirror):
    import torch
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    rho = torch.ones(32**3, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.DfError) as ei:
        binding.force_level_noalloc(rho.data_ptr(), (16, 16, 16), 8, (-1, -1, -1),
                                    (0.125,) * 3, off, ext, 1.0, 0.1, 1.0, out.data_ptr(), None,
                                    mirror=mirror)
    assert ei.value.code == binding.DF_EINVAL
