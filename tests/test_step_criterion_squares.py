"""The block-step criterion is compared on squares (CPU).

The step choice compares the criterion da = sqrt_rn(y) only with powers of two
p (halving while p > da, doubling while da >= 2h).  The kernels compare y with
p^2 instead, which takes the same decisions exactly: p^2 is exact, and no
double lies in the half ulp below p^2 that would make sqrt_rn round up to p.
This checks that equivalence with IEEE square roots (numpy's are correctly
rounded) at and around every boundary, and on random values.
"""
import numpy as np


def _decisions(y, p):
    da = np.sqrt(y)
    return (p > da), (y < p * p)


def test_square_comparison_equals_the_square_root_comparison():
    rng = np.random.default_rng(7)
    for e in range(-60, 61, 3):
        p = np.float64(2.0) ** e
        p2 = p * p
        # the boundary itself and its neighbours, a few ulps either side
        ys = [p2]
        lo = hi = p2
        for _ in range(8):
            lo = np.nextafter(lo, 0.0)
            hi = np.nextafter(hi, np.inf)
            ys += [lo, hi]
        # random values across two decades around p^2
        ys += list(p2 * np.exp(rng.uniform(-2.3, 2.3, 200)))
        ys = np.array(ys, dtype=np.float64)
        a, b = _decisions(ys, p)
        assert np.array_equal(a, b), (e, ys[a != b])


def test_the_half_ulp_below_p_squared_holds_no_double():
    # sqrt_rn(y) rounds up to p only for y >= p^2 (1 - 2^-53 + 2^-108); the
    # largest double below p^2 is p^2 (1 - 2^-53), just under that
    for e in (-40, -7, 0, 5, 40):
        p = np.float64(2.0) ** e
        below = np.nextafter(p * p, 0.0)
        assert np.sqrt(below) < p
        assert np.sqrt(p * p) == p
