"""The allocation-free force entry point agrees with the context's force reduction.

df_force_level_noalloc serves callers that cannot call cudaMalloc (device memory
fully reserved by another allocator, loops that cannot take cudaMalloc's implicit
synchronisation, sandboxed plug-ins).  It keeps its scratch in a fixed device array
shared by every call, so this test checks two calls in a row, on different states,
against df_force_now, and that oversize input is rejected.  Collected last: it runs
alone in a fresh process as well as after every other test.
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


def _level_geometry(sim, level, half):
    n = sim.n
    dx = [2 * half / 2**level / n[d] for d in range(3)]
    lo = [-half / 2**level] * 3
    return n, lo, dx


def _noalloc_total(sim, half, params, stream):
    """sum over levels of the allocation-free per-level force"""
    import torch
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    total = np.zeros(3)
    for l in range(sim.n_levels):
        rho = torch.from_numpy(sim.get_full(l, 0).ravel().copy()).cuda()
        n, lo, dx = _level_geometry(sim, l, half)
        child_off = child_n = None
        if l + 1 < sim.n_levels:
            child_off = [n[d] // 4 for d in range(3)]
            child_n = [n[d] // 2 for d in range(3)]
        binding.force_level_noalloc(rho.data_ptr(), n, sim.G, lo, dx, child_off, child_n,
                                    params["GM"], params["eps"], params["rho0"],
                                    out.data_ptr(), stream)
        torch.cuda.current_stream().synchronize()
        total += out.cpu().numpy()
    return total


@pytest.mark.parametrize("n_levels", [1, 3])
def test_noalloc_force_matches_context_force_twice(n_levels):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    half = 6.0
    p = I.base_params(GM=0.013, eps=0.2, chi=0.5, L=0.05, lum_sigma=0.25, mach=0.7)
    sim = binding.Sim(n_levels, 24, (-half,) * 3, (half,) * 3, I.DEFAULT_G, p)
    for call in range(2):
        sim.step(3 + 4 * call)  # a different state for each call
        ref = sim.force_now()
        got = _noalloc_total(sim, half, p, stream)
        assert np.abs(got - ref).max() <= TOL * np.abs(ref).max(), (call, got, ref)
        assert np.abs(ref).max() > 0
    sim.close()


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
