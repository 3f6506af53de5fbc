"""Host-side checks of FP32 identities the CUDA kernels rely on (no GPU).

The kernels form the uniform u = (2 (w >> 9) + 1) 2^-24 of a Philox word w
(the counter-stream uniform of the oracle's orc_u24) without an
integer-to-float conversion: the 23 bits w >> 9 become the mantissa of
1.m in [1, 2), and u = 1.m - (1 - 2^-24).  The difference m 2^-23 + 2^-24 is
an odd multiple of 2^-24 below 1, so it is representable and the IEEE
round-to-nearest subtraction returns it exactly.  These tests check the
identity for every mantissa in IEEE single precision (numpy float32 follows
the same rounding as the GPU's FP32 add)."""
import numpy as np


def test_uniform_from_mantissa_bits_is_exact_for_every_mantissa():
    m = np.arange(1 << 23, dtype=np.uint32)
    one_m = (m | np.uint32(0x3F800000)).view(np.float32)
    c = np.float32(1.0 - 2.0 ** -24)
    assert float(c) == 1.0 - 2.0 ** -24  # the constant itself is exact
    got = one_m - c
    assert got.dtype == np.float32
    # the definition, in FP64 (exact) and then to FP32 (exact as well)
    want = ((2.0 * m.astype(np.float64) + 1.0) * 2.0 ** -24).astype(np.float32)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    assert got.min() == np.float32(2.0 ** -24) and got.max() == np.float32(1.0 - 2.0 ** -24)


def test_uniform_from_mantissa_bits_matches_the_word_layout():
    # a few words whose uniform is known by hand: the low 9 bits are dropped
    w = np.array([0, 0x1FF, 0x200, 0xFFFFFFFF, 0x80000000], dtype=np.uint32)
    one_m = ((w >> np.uint32(9)) | np.uint32(0x3F800000)).view(np.float32)
    got = (one_m - np.float32(1.0 - 2.0 ** -24)).astype(np.float64)
    want = np.array([2.0 ** -24, 2.0 ** -24, 3 * 2.0 ** -24, 1.0 - 2.0 ** -24, 0.5 + 2.0 ** -24])
    assert np.array_equal(got, want)
