"""The block-step criterion is compared on squares (CPU).

The step choice compares the criterion da = sqrt_rn(y) only with powers of two
p (halving while p > da, doubling while da >= 2h).  The kernels compare y with
p^2 instead, which takes the same decisions exactly: p^2 is exact, and no
double lies in the half ulp below p^2 that would make sqrt_rn round up to p.
This checks that equivalence with IEEE square roots (numpy's are correctly
rounded) at and around every boundary, and on random values, in FP64 (the
FP64 path) and in FP32 (the F32C path's corrector takes the criterion in FP32,
for steps from 2^-60 to 2^60, where p^2 is a normal float).
"""
import numpy as np
import pytest


def _decisions(y, p):
    da = np.sqrt(y)
    return (p > da), (y < p * p)


@pytest.mark.parametrize("dtype,emax", [(np.float64, 60), (np.float32, 60)])
def test_square_comparison_equals_the_square_root_comparison(dtype, emax):
    rng = np.random.default_rng(7)
    for e in range(-emax, emax + 1, 3):
        p = dtype(2.0) ** e
        p2 = p * p
        # the boundary itself and its neighbours, a few ulps either side
        ys = [p2]
        lo = hi = p2
        for _ in range(8):
            lo = np.nextafter(lo, dtype(0.0))
            hi = np.nextafter(hi, dtype(np.inf))
            ys += [lo, hi]
        # random values across two decades around p^2
        ys += list(p2 * np.exp(rng.uniform(-2.3, 2.3, 200)).astype(dtype))
        ys = np.array(ys, dtype=dtype)
        a, b = _decisions(ys, p)
        assert p2 == dtype(2.0) ** (2 * e)  # exact, and a normal number
        assert np.array_equal(a, b), (e, ys[a != b])


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_the_half_ulp_below_p_squared_holds_no_value(dtype):
    # sqrt_rn(y) rounds up to p only for y >= p^2 (1 - u + u^2/4) (u the unit
    # roundoff, 2^-53 or 2^-24); the largest value below p^2 is p^2 (1 - u),
    # just under that
    for e in (-40, -7, 0, 5, 40):
        p = dtype(2.0) ** e
        below = np.nextafter(p * p, dtype(0.0))
        assert np.sqrt(below) < p
        assert np.sqrt(p * p) == p
