"""The error model behind the gradient parity bar (no GPU): a float-pair
("double-float") sum of exact products, TwoProd by FMA and Knuth's TwoSum
(Dekker 1971; Ogita, Rump & Oishi 2005), restated in IEEE FP32 with numpy and
checked against an exact rational sum.  One lane of the gradient kernels sums
about 455 rows this way on the 1,048,576-row workload; the parity bar is
1e-12 of sum_i |a_i| |r_i|."""
from fractions import Fraction

import numpy as np

F32 = np.float32


def _two_sum(a, b):
    s = F32(a + b)
    bb = F32(s - a)
    return s, F32(F32(a - F32(s - bb)) + F32(b - bb))


def _pair_dot(a, rh, rl):
    """(hi, lo) = sum_i a_i (rh_i + rl_i): each a_i * rh_i split exactly into
    an FP32 pair (the product of two FP32 values is exact in FP64), TwoSum
    into hi, the low parts and a_i * rl_i into lo in FP32."""
    hi, lo = F32(0), F32(0)
    for ai, hi_i, lo_i in zip(a, rh, rl):
        p64 = float(ai) * float(hi_i)
        p = F32(p64)
        pe = F32(p64 - float(p))
        hi, e = _two_sum(hi, p)
        lo = F32(lo + F32(e + pe))
        lo = F32(float(ai) * float(lo_i) + float(lo))
    return hi, lo


def test_float_pair_lane_sum_is_far_inside_the_gradient_bar():
    """Over 50 draws of 455 N(0,1) entries and 0.1 N(0,1) residuals, the pair
    sum errs by at most 1e-13 of sum |a_i r_i| (ten times inside the 1e-12
    bar), while the same sum in plain FP32 errs by more than 1e-9 (so a
    kernel that lost its low words would fail the bar)."""
    rng = np.random.default_rng(0)
    L = 455
    worst_pair, worst_f32 = 0.0, 0.0
    for _ in range(50):
        a = rng.standard_normal(L).astype(F32)
        r = 0.1 * rng.standard_normal(L)
        rh = r.astype(F32)
        rl = (r - rh.astype(np.float64)).astype(F32)
        exact = sum(Fraction(float(x)) * (Fraction(float(h)) + Fraction(float(l)))
                    for x, h, l in zip(a, rh, rl))
        scale = float(np.abs(a.astype(np.float64) * r).sum())
        hi, lo = _pair_dot(a, rh, rl)
        worst_pair = max(worst_pair,
                         abs(float(Fraction(float(hi)) + Fraction(float(lo)) - exact)) / scale)
        s32 = F32(0)
        for x, h in zip(a, rh):
            s32 = F32(s32 + F32(x * h))
        worst_f32 = max(worst_f32, abs(float(Fraction(float(s32)) - exact)) / scale)
    assert worst_pair < 1e-13
    assert worst_f32 > 1e-9
