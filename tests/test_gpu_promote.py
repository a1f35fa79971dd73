"""The exact FP32 -> FP64 promotion that the FP64 combines run on the integer pipe (the
averages d*_k and y_0 of the FP32-state combine, Sec. 2.1 / Sec. 3.2, summed in FP64) against
the device's conversion instruction, over every float bit pattern.

The library's self-test entry point compares the two on the GPU for a range of bit patterns.
Finite values, signed zeros, subnormals and infinities agree bit for bit, and so do quiet NaNs
(sign and payload kept).  A signalling NaN differs in the quiet bit alone: the conversion sets
it, the promotion keeps the float's bits; the combine's FMA turns either into a NaN, so no
combine result depends on it.  2 x (2^22 - 1) float patterns are signalling NaNs.
"""
import pytest
import torch

from paper_1907_11771_gb300 import binding as B

pytestmark = pytest.mark.gpu
SNAN_PER_SIGN = (1 << 22) - 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1907_11771_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_promotion_matches_the_conversion_on_every_float():
    total = [0, 0, 0]
    chunk = 1 << 30
    for first in range(0, 1 << 32, chunk):
        for i, n in enumerate(B.gbs_selftest_f32_to_f64(first, chunk)):
            total[i] += n
    assert total == [0, 0, 2 * SNAN_PER_SIGN], total


@pytest.mark.parametrize("first,count,quiet_bit_only", [
    (0, 1, 0),                                   # +0
    (0x00000001, 0x007fffff, 0),                 # the positive subnormals
    (0x7f7fffff, 2, 0),                          # the largest finite, +infinity
    (0x7f800001, SNAN_PER_SIGN, SNAN_PER_SIGN),  # the positive signalling NaNs
    (0x7fc00000, 1 << 22, 0),                    # the positive quiet NaNs
    (0x80000000, 1, 0),                          # -0
    (0x80000001, 0x007fffff, 0),                 # the negative subnormals
    (0xff800000, 1, 0),                          # -infinity
    (0xff800001, SNAN_PER_SIGN, SNAN_PER_SIGN),  # the negative signalling NaNs
    ((1 << 32) - 1, 1, 0),                       # the last pattern, a quiet NaN
    (5, 0, 0),                                   # an empty range
])
def test_promotion_on_the_special_ranges(first, count, quiet_bit_only):
    assert B.gbs_selftest_f32_to_f64(first, count) == (0, 0, quiet_bit_only)


def test_selftest_rejects_ranges_outside_the_float_patterns():
    with pytest.raises(B.GbsError):
        B.gbs_selftest_f32_to_f64((1 << 32) - 1, 2)
    with pytest.raises(B.GbsError):
        B.gbs_selftest_f32_to_f64((1 << 32) + 1, 0)
