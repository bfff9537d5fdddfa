"""The hot path's contract calls, through the C ABI on the GPU: df_create_levels
(with the caller's allocator callbacks), df_set_params, df_step with its time
output, df_force, df_get_field, df_destroy, and for pools df_pool_create /
admit / step / df_pool_force / release -- each result against the FP64 oracle
(Sec. 3 and Sec. 3.4 set-up)."""
import ctypes as C

import numpy as np
import pytest

from oracle import Oracle
from paper_1812_03191_gb300 import binding
from paper_1812_03191_gb300 import inputs as I

from test_gpu_parity import TOL, force_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1812_03191_gb300 import build as B
    B.build()
    binding.load()


class _View:
    """the geometry attributes force_bound reads"""

    def __init__(self, n_levels, n, lo, hi):
        self.n_levels, self.n, self.n0, self.lo, self.hi = n_levels, (n,) * 3, (n,) * 3, lo, hi


def _check(lib, rc):
    assert rc == binding.DF_OK, lib.df_last_error().decode()


def test_create_levels_step_force_destroy_against_the_oracle():
    import torch
    lib = binding.load()
    nl, N, half = 3, 24, 6.0
    lo, hi = (-half,) * 3, (half,) * 3
    p = I.base_params(GM=0.01, eps=0.125, chi=1.0, L=0.05, lum_sigma=0.125, mach=0.5)
    live = {}

    def alloc(nbytes, user):
        ptr = torch.cuda.caching_allocator_alloc(int(nbytes))
        live[ptr] = nbytes
        return ptr

    def free(ptr, user):
        live.pop(ptr)
        torch.cuda.caching_allocator_delete(ptr)

    fa, ff = binding._ALLOC_FN(alloc), binding._FREE_FN(free)
    h = C.c_void_p()
    stream = torch.cuda.current_stream().cuda_stream
    _check(lib, lib.df_create_levels(C.byref(h), nl, N, (C.c_double * 3)(*lo),
                                     (C.c_double * 3)(*hi), binding.DF_FP64, 0,
                                     C.c_void_p(stream), C.cast(fa, C.c_void_p),
                                     C.cast(ff, C.c_void_p), None))
    assert live, "the context took its device memory from the callbacks"
    _check(lib, lib.df_set_params(h, C.byref(binding.Params.from_dict(p))))
    orc = Oracle(nl, N, lo, hi, binding_ghost(), p)
    t = C.c_double()
    _check(lib, lib.df_step(h, 6, C.byref(t)))
    orc.step(6)
    assert abs(t.value - orc.t) <= 1e-13 * orc.t
    worst = rho_err = 0.0
    for l in range(nl):
        for f in range(5):
            a = np.empty(N**3)
            _check(lib, lib.df_get_field(h, l, f, a.ctypes.data_as(C.POINTER(C.c_double))))
            e = np.abs(a - orc.get_field(l, f).ravel()).max() / (1.0 if f < 2 else 0.5)
            worst = max(worst, e)
            if f == 0:
                rho_err = max(rho_err, e)
    assert worst <= TOL, worst
    F = (C.c_double * 3)()
    along = C.c_double()
    _check(lib, lib.df_force(h, F, C.byref(along)))
    Fo = orc.force()
    bound = force_bound(_View(nl, N, lo, hi), orc, p, rho_err)
    assert np.abs(np.array(F[:]) - Fo).max() <= bound
    assert abs(along.value - F[0]) <= 1e-15 * abs(F[0])  # wind along -x: motion +x
    # an asynchronous step (no time output) continues the same run
    _check(lib, lib.df_step(h, 2, None))
    orc.step(2)
    _check(lib, lib.df_step(h, 0, C.byref(t)))
    assert abs(t.value - orc.t) <= 1e-13 * orc.t
    _check(lib, lib.df_destroy(h))
    assert not live, "every block went back through the callbacks"
    orc.close()


def binding_ghost():
    return 8  # DF_DEFAULT_GHOST, the ghost width df_create_levels uses


def test_pool_force_per_slot_against_the_oracle():
    lib = binding.load()
    runs = [(2, 24, 6.0, dict(mach=0.4, chi=0.7, GM=0.01, eps=0.25)),
            (3, 24, 6.0, dict(mach=1.3, chi=0.3, L=0.05, lum_sigma=0.2, GM=0.01, eps=0.2))]
    pool = binding.Pool(1 << 34)
    slots, orcs = [], []
    for nl, n, half, over in runs:
        p = I.base_params(**over)
        slots.append(pool.admit(nl, n, (-half,) * 3, (half,) * 3, I.DEFAULT_G, p))
        orcs.append(Oracle(nl, n, (-half,) * 3, (half,) * 3, I.DEFAULT_G, p))
    _check(lib, lib.df_pool_step(pool.h, 5))
    for (nl, n, half, over), slot, orc in zip(runs, slots, orcs):
        orc.step(5)
        p = I.base_params(**over)
        F = (C.c_double * 3)()
        t = C.c_double()
        _check(lib, lib.df_pool_force(pool.h, slot, F, C.byref(t)))
        assert abs(t.value - orc.t) <= 1e-13 * orc.t
        rho_err = max(np.abs(pool.get_field(slot, l, 0) - orc.get_field(l, 0)).max()
                      for l in range(nl))
        assert rho_err <= TOL
        Fo = orc.force()
        lo, hi = (-half,) * 3, (half,) * 3
        assert np.abs(np.array(F[:]) - Fo).max() <= force_bound(_View(nl, n, lo, hi), orc, p,
                                                                 rho_err)
    pool.release(slots[0])
    F = (C.c_double * 3)()
    assert lib.df_pool_force(pool.h, slots[0], F, None) == binding.DF_EINVAL
    pool.close()
