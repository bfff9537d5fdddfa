"""The double-float arithmetic of the FP64 stencils (csrc/df64.h: Knuth's two-sum,
Dekker's fast two-sum and long division, the fused-multiply-add product), checked on
the CPU against FP64 on two million operand pairs over 40 decades (compiled as host
code with nvcc; no GPU needed).  The device's reciprocal estimate is checked on the
GPU (tests/test_gpu_df64.py)."""
from test_index_math_cpu import _run_check


def test_double_float_operations_within_their_bounds(tmp_path):
    _run_check(tmp_path, "df64_check")
