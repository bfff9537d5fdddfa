"""Device memory from the caller's allocator (df_set_allocator): a context and a pool
created while PyTorch's caching allocator is installed hold their buffers in torch's
accounting, give them back when closed, and compute the same bits as with
cudaMalloc."""
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


def _params():
    return I.base_params(GM=0.02, eps=0.3, chi=0.4, L=0.03, lum_sigma=0.3, mach=0.9)


def test_torch_allocator_holds_the_runs_memory():
    import torch
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    lo, hi = (-6.0,) * 3, (6.0,) * 3
    plain = binding.Sim(3, 24, lo, hi, I.DEFAULT_G, _params())
    assert torch.cuda.memory_allocated() == base  # cudaMalloc: outside torch's books
    binding.use_torch_allocator(True)
    try:
        sim = binding.Sim(3, 24, lo, hi, I.DEFAULT_G, _params())
        pool = binding.Pool(1 << 30, precision=binding.DF_FP32_STATE)
        slot = pool.admit(2, 32, lo, hi, I.DEFAULT_G, _params())
    finally:
        binding.use_torch_allocator(False)
    held = torch.cuda.memory_allocated() - base
    need = (binding.run_bytes(3, 24, I.DEFAULT_G, binding.DF_FP64)
            + binding.run_bytes(2, 32, I.DEFAULT_G, binding.DF_FP32_STATE))
    assert held >= need, (held, need)
    for s in (plain, sim):
        s.step(5)
    pool.step(5)
    for l in range(3):
        for f in range(5):
            assert np.array_equal(plain.get_field(l, f), sim.get_field(l, f)), (l, f)
    assert np.array_equal(plain.force()[0], sim.force()[0])
    assert pool.query()[slot, 5] == 0
    # the plans built by the first steps came from torch too; a context created
    # after the switch back uses cudaMalloc again
    stepped = torch.cuda.memory_allocated()
    assert stepped > base + held - 1
    again = binding.Sim(2, 24, lo, hi, I.DEFAULT_G, _params())
    again.step(2)
    assert torch.cuda.memory_allocated() == stepped
    for s in (sim, again, plain):
        s.close()
    pool.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base


def test_allocator_arguments_are_checked():
    lib = binding.load()
    import ctypes
    fn = binding._ALLOC_FN(lambda n, u: None)
    assert lib.df_set_allocator(ctypes.cast(fn, ctypes.c_void_p), None, None) == binding.DF_EINVAL
    assert lib.df_set_allocator(None, None, None) == binding.DF_OK
