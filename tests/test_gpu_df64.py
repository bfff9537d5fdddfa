"""The double-float arithmetic of the FP64 stencils on the device (the hardware
reciprocal estimate included) against FP64: conversion, sum, product and quotient,
each within its bound, on operands spread over 40 decades; the unnormalised product
and quotient within the same bounds, their low parts within 2^-21 of their high
parts, and a sum taking the unnormalised product within its bound."""
import numpy as np
import pytest

from paper_1812_03191_gb300 import binding

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1812_03191_gb300 import build as B
    B.build()
    binding.load()


def test_double_float_operations_on_the_device():
    rng = np.random.default_rng(23)
    n = 1 << 20

    def operands():
        return (rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-20, 2, n)
                * (1 + rng.random(n)))

    w = binding.check_df64(operands(), operands())
    print("worst error / bound (conversion, sum, product, quotient, unnormalised "
          "product, unnormalised quotient, their low parts, sum with one):", w)
    assert np.all(w <= 1.0), w


def test_fp64_state_values_are_doubles_of_47_bits():
    """The FP64 state as stored: a value written in comes back within 2^-44 of its
    deviation from the background (cut to 47 significant bits: to a pair, then lo onto
    its grid, each toward zero), and a state read out and written back is unchanged bit
    for bit (the stored values are doubles)."""
    from paper_1812_03191_gb300 import inputs as I
    p = I.base_params()
    sim = binding.Sim(1, 16, (-4.0,) * 3, (4.0,) * 3, I.DEFAULT_G, p)
    rng = np.random.default_rng(5)
    bg = [p["rho0"], sim.get_full(0, 1).mean(), -p["mach"] * p["cs"], 0.0, 0.0]
    for f in range(5):
        dev = rng.choice([-1.0, 1.0], sim.full_shape()) * 10.0 ** rng.uniform(
            -12, 0, sim.full_shape())
        sim.set_full(0, f, bg[f] + dev)
        got = sim.get_full(0, f) - bg[f]
        # the background is removed and added back in FP64, on the device and here:
        # three roundings of half an ulp of |bg| + |dev|
        slack = 2.0**-53 * (abs(bg[f]) + np.abs(dev))
        assert np.all(np.abs(got - dev) <= 2.0**-44 * np.abs(dev) + 3 * slack), f
    st, t = sim.get_state()
    sim.set_state(st, t)
    st2, t2 = sim.get_state()
    assert t2 == t and np.array_equal(st, st2)
