"""The shortcut of the device-side exact decision (exact_within in
csrc/egm_internal.cuh), restated with Python floats, never contradicts the
definition it stands in for.

The definition (Eq. 3 / Eq. 4 as the brute force evaluates it): with
num = |RN(RN(RN(a x) + RN(b y)) + c)| and N = RN(sqrt(RN(RN(a a) + RN(b b)))),
a reference is a candidate when RN(num / N) <= eps.  The shortcut compares
lhs = RN(num num) with rhs = RN(RN(eps eps) S) widened by 2^-48 either way and
leaves everything in between (and outside the normal range) to the
definition.  Python floats are IEEE doubles with round-to-nearest and a
correctly rounded math.sqrt, so both sides here round exactly as the device
does.  Cases sit on the boundary: eps equal to the quotient, one ulp either
side, and a few ulps either side.
"""
import math
import random

import pytest

M_LO = 1.0 - 2.0 ** -48
M_HI = 1.0 + 2.0 ** -48


def definition(a, b, c, x, y, eps):
    num = abs((a * x + b * y) + c)
    return num / math.sqrt(a * a + b * b) <= eps


def shortcut(a, b, c, x, y, eps):
    """True / False when the shortcut decides, None when it defers."""
    num = abs((a * x + b * y) + c)
    S = a * a + b * b
    if 1e-140 <= eps <= 1e140 and num <= 1e145:
        lhs = num * num
        rhs = (eps * eps) * S
        if 1e-290 <= rhs <= 1e290:
            if lhs <= rhs * M_LO:
                return True
            if lhs >= rhs * M_HI:
                return False
    return None


def _cases(rng, n):
    for _ in range(n):
        # a line through the image of a plausible F and point, in pixels
        a = rng.uniform(-1, 1) * 10.0 ** rng.uniform(-6, 1)
        b = rng.uniform(-1, 1) * 10.0 ** rng.uniform(-6, 1)
        c = rng.uniform(-1, 1) * 10.0 ** rng.uniform(-4, 3)
        x = rng.uniform(-6000, 6000)
        y = rng.uniform(-4000, 4000)
        if a == 0.0 and b == 0.0:
            continue
        q = abs((a * x + b * y) + c) / math.sqrt(a * a + b * b)
        if not (q > 0.0 and math.isfinite(q)):
            continue
        for eps in (q, math.nextafter(q, math.inf), math.nextafter(q, 0.0),
                    q * (1 + 2.0 ** -50), q * (1 - 2.0 ** -50), q * (1 + 2.0 ** -45), q * (1 - 2.0 ** -45),
                    q * (1 + 1e-9), q * (1 - 1e-9), q * 1.5, q * 0.5):
            yield a, b, c, x, y, eps


def test_shortcut_agrees_with_definition_on_the_boundary():
    rng = random.Random(20260318)
    decided = 0
    total = 0
    for a, b, c, x, y, eps in _cases(rng, 20000):
        s = shortcut(a, b, c, x, y, eps)
        total += 1
        if s is None:
            continue
        decided += 1
        assert s == definition(a, b, c, x, y, eps), (a, b, c, x, y, eps)
    # away from the last few ulps the shortcut decides
    assert decided > 0.5 * total


@pytest.mark.parametrize("scale", [1e-150, 1e-100, 1.0, 1e100, 1e150])
def test_shortcut_defers_or_agrees_at_extreme_scales(scale):
    rng = random.Random(int(abs(math.log10(scale))) + 7)
    for a, b, c, x, y, eps in _cases(rng, 2000):
        a2, b2, c2 = a * scale, b * scale, c * scale
        if not all(math.isfinite(v) for v in (a2, b2, c2)) or (a2 == 0.0 and b2 == 0.0):
            continue
        try:
            ref = definition(a2, b2, c2, x, y, eps)
        except (ZeroDivisionError, OverflowError):
            continue
        s = shortcut(a2, b2, c2, x, y, eps)
        assert s is None or s == ref
