"""The integer bit recipes the mixed-form kernels use in place of FP64-pipe
instructions, restated in NumPy and checked against IEEE 754 conversions on
the host.

f32 -> f64 widening (`f32_to_f64` in the CUDA source): for a normal float,
rebias the exponent by 1023 - 127 = 896 and move the 23-bit significand to
the top of the 52-bit one; zero keeps its sign; subnormal, infinite and NaN
inputs go to the hardware conversion (not restated here).  The sign, the
exponent and the significand land in disjoint bit fields, so checking every
significand under a few exponents and every exponent under many significands,
with both signs, covers every input.
"""
import numpy as np


def _widen(u):
    u = u.astype(np.uint64)
    e = (u >> np.uint64(23)) & np.uint64(0xFF)
    m = u & np.uint64(0x7FFFFF)
    sign = u & np.uint64(0x80000000)
    normal = (e >= 1) & (e <= 0xFE)
    hi = np.where(normal, sign | ((e + np.uint64(896)) << np.uint64(20)) | (m >> np.uint64(3)), sign)
    lo = np.where(normal, (m << np.uint64(29)) & np.uint64(0xFFFFFFFF), np.uint64(0))
    handled = normal | ((u & np.uint64(0x7FFFFFFF)) == 0)
    return (hi << np.uint64(32)) | lo, handled


def _check(u):
    bits, handled = _widen(u)
    ref = u.astype(np.uint32).view(np.float32)[handled].astype(np.float64).view(np.uint64)
    assert np.array_equal(bits[handled], ref)
    return handled


def test_f32_to_f64_widening_every_significand():
    m = np.arange(1 << 23, dtype=np.uint64)
    for sign in (0, 1):
        for e in (1, 100, 127, 200, 254):
            assert _check((sign << 31) | (e << 23) | m).all()


def test_f32_to_f64_widening_every_exponent_zero_and_specials():
    rng = np.random.default_rng(0)
    m = np.unique(np.r_[0, 1, 0x7FFFFF, 0x400000, rng.integers(0, 1 << 23, 4096)]).astype(np.uint64)
    for sign in (0, 1):
        for e in range(256):
            h = _check((np.uint64(sign << 31) | np.uint64(e << 23)) | m)
            if 1 <= e <= 254:
                assert h.all()
            elif e == 0:
                assert h[m == 0].all() and not h[m != 0].any()   # zero handled, subnormals to hardware
            else:
                assert not h.any()                                # inf / nan to hardware
