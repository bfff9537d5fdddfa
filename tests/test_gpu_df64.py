"""The double-float arithmetic of the FP64 stencils on the device (the hardware
reciprocal estimate included) against FP64: conversion, sum, product and quotient,
each within its bound, on operands spread over 40 decades."""
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
    print("worst error / bound (conversion, sum, product, quotient):", w)
    assert np.all(w <= 1.0), w
