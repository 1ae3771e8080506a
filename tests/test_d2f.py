"""The integer-pipe double -> float conversion of the prep kernel (d2f in
csrc/geom.cu), restated step by step with numpy integers, equals IEEE 754
round-to-nearest-even conversion (numpy's float64 -> float32 cast) wherever
it does not hand the value to the hardware conversion: ties to even and
to odd, carries out of the fraction into the exponent, the ends of the
normal float range and the overflow to infinity.
"""
import numpy as np


def d2f_steps(d):
    """The kernel's steps; None where it takes the hardware conversion."""
    u = np.asarray(d, np.float64).view(np.uint64)
    hi = (u >> np.uint64(32)).astype(np.uint32)
    lo = (u & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    e = (hi >> np.uint32(20)) & np.uint32(0x7FF)
    other = (e - np.uint32(897)) > np.uint32(253)  # unsigned wrap, as on the device
    f = ((hi & np.uint32(0x80000000)) | ((e - np.uint32(896)) << np.uint32(23))
         | ((hi & np.uint32(0xFFFFF)) << np.uint32(3)) | (lo >> np.uint32(29)))
    rem = lo & np.uint32(0x1FFFFFFF)
    up = (rem > np.uint32(0x10000000)) | ((rem == np.uint32(0x10000000)) & ((f & np.uint32(1)) == 1))
    f = f + up.astype(np.uint32)
    return f.view(np.float32), other


def _check(d):
    d = np.asarray(d, np.float64)
    got, other = d2f_steps(d)
    with np.errstate(over="ignore"):
        want = d.astype(np.float32)
    sel = ~other
    assert sel.any()
    np.testing.assert_array_equal(got[sel].view(np.uint32), want[sel].view(np.uint32))
    return other


def test_random_doubles_in_the_float_range():
    rng = np.random.default_rng(11)
    m = rng.uniform(-1.0, 1.0, 200000)
    d = m * np.exp2(rng.integers(-126, 128, m.size).astype(np.float64))
    other = _check(d)
    assert other.mean() < 0.01


def test_ties_and_carries():
    rng = np.random.default_rng(12)
    # float32 values with the 29 dropped bits set to exactly half, just below and just above
    f = rng.integers(0x00800000, 0x7F7FFFFF, 50000, dtype=np.uint32).view(np.float32).astype(np.float64)
    u = f.view(np.uint64)
    for low in (0x10000000, 0x0FFFFFFF, 0x10000001, 0x1FFFFFFF, 0x00000001):
        _check((u | np.uint64(low)).view(np.float64))
        _check(-(u | np.uint64(low)).view(np.float64))
    # all fraction bits set: the rounding carries into the exponent
    ones = np.array([np.float32(1.9999999), np.float32(3.9999998), np.float32(1.1754942e-38) * 2], np.float64)
    _check((ones.view(np.uint64) | np.uint64(0x1FFFFFFF)).view(np.float64))


def test_range_ends():
    fmax = float(np.finfo(np.float32).max)
    tiny = float(np.finfo(np.float32).tiny)
    half_ulp_max = 2.0 ** 103  # half an ulp of the largest float
    cases = [fmax, -fmax, np.nextafter(fmax + half_ulp_max, 0.0), fmax + half_ulp_max,
             np.nextafter(fmax + half_ulp_max, np.inf), tiny, -tiny, np.nextafter(tiny, np.inf),
             1.0, -1.0, 0.5, 3024.0, 6047.999999999, 1e-30, 1e30]
    other = _check(cases)
    # the tie above the largest float rounds to even, which is infinity
    got, _ = d2f_steps([fmax + half_ulp_max])
    assert np.isinf(got[0])
    # zeros, subnormal results and values beyond the float range go to the hardware
    _, o = d2f_steps([0.0, -0.0, tiny / 2, 1e-300, 2.0 ** 128, 1e300, np.inf, np.nan])
    assert o.all() and not other[:5].any()
