"""The error bound of the emulated FP64 product (FP32 pairs), checked in exact
arithmetic on the CPU.

The emulated variants sum each row as an FP32 pair: values and x are split
into hi + lo (hi rounded half-up on the magnitude to 24 bits, lo the rest
rounded to nearest FP32), and every term takes one double-word step
(dw::dw_fma: TwoProduct plus cross products, TwoSum into the high word,
the rest into the low word, Fast2Sum).  The stated bound, for a row of k <= 48
terms with every nonzero |a|, |x| in [2^-45, 2^60], is

    |y - sum_j a_j x_j| <= (5.2 k + 18) 2^-48 sum_j |a_j x_j|   (< 9.6e-13).

Here every FP32 operation of that step sequence is carried out as an exact
rational followed by round-to-nearest-even to FP32 (subnormals included),
on rows built to cancel (random signs, terms of equal size with opposite
signs, magnitudes spread over the whole window), and the result is compared
with the exact sum.  A planted weaker step (the low word dropped) must break
the bound.
"""
from fractions import Fraction as Q
import math

import pytest

import synth

U2 = Q(1, 2 ** 48)


def rn32(q: Q) -> Q:
    """Round a rational to the nearest FP32 number, ties to even (gradual
    underflow; no overflow occurs in these rows)."""
    if q == 0:
        return Q(0)
    sign = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Q(2) ** e > a:
        e -= 1
    e = max(e, -126)
    ulp = Q(2) ** (e - 23)
    m = a / ulp
    fl = math.floor(m)
    r = m - fl
    if r > Q(1, 2) or (r == Q(1, 2) and fl % 2 == 1):
        fl += 1
    return sign * fl * ulp


def split(v: float):
    """hi = v rounded half-up on the magnitude to 24 significant bits, lo =
    RN32(v - hi), as the library splits values and x."""
    q = Q(v)
    if q == 0:
        return Q(0), Q(0)
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Q(2) ** e > a:
        e -= 1
    ulp = Q(2) ** (e - 23)
    hi = math.floor(a / ulp + Q(1, 2)) * ulp
    hi = hi if q > 0 else -hi
    return hi, rn32(q - hi)


def two_sum(a, b):
    s = rn32(a + b)
    bb = rn32(s - a)
    e = rn32(rn32(a - rn32(s - bb)) + rn32(b - bb))
    return s, e


def fast_two_sum(a, b):
    s = rn32(a + b)
    return s, rn32(b - rn32(s - a))


def dw_step(sh, sl, a, x, keep_low=True):
    ph = rn32(a[0] * x[0])
    pe = rn32(a[0] * x[0] - ph)
    pe = rn32(a[0] * x[1] + pe)
    pe = rn32(a[1] * x[0] + pe)
    s, e = two_sum(sh, ph)
    t = rn32(sl + rn32(e + pe)) if keep_low else Q(0)
    return fast_two_sum(s, t)


def row_error(avals, xvals, keep_low=True):
    sh = sl = Q(0)
    for a, x in zip(avals, xvals):
        sh, sl = dw_step(sh, sl, split(a), split(x), keep_low)
    y = float(sh + sl)                      # both exact in FP64; one RN64
    exact = sum(Q(a) * Q(x) for a, x in zip(avals, xvals))
    scale = sum(abs(Q(a) * Q(x)) for a, x in zip(avals, xvals))
    return abs(Q(y) - exact), scale


def bound(k, scale):
    return (Q(52, 10) * k + 18) * U2 * scale


def rows(seed, count):
    rng = synth.Rng(seed, 5)
    for r in range(count):
        k = int(rng.integers(1, 1, 49)[0])
        kind = r % 4
        if kind == 0:        # random signs, magnitudes over the whole window
            ea = rng.uniform(k, -45, 59.9)
            ex = rng.uniform(k, -45, 59.9)
        elif kind == 1:      # products of one size: heavy cancellation
            ea = rng.uniform(k, -5, 5)
            ex = -ea + rng.uniform(k, -0.01, 0.01)
        elif kind == 2:      # small terms around an early large one
            ea = rng.uniform(k, -40, -20)
            ex = rng.uniform(k, -5, 5)
            ea[0] = 30.0
        else:                # near the top of the window
            ea = rng.uniform(k, 50, 59.9)
            ex = rng.uniform(k, 50, 59.9)
        sa = rng.unit(k) < 0.5
        sx = rng.unit(k) < 0.5
        a = [(-1.0 if s else 1.0) * 2.0 ** float(e) for s, e in zip(sa, ea)]
        x = [(-1.0 if s else 1.0) * 2.0 ** float(e) for s, e in zip(sx, ex)]
        if kind == 1 and k > 1:   # exact pairs of opposite terms
            for j in range(1, k, 2):
                a[j], x[j] = -a[j - 1], x[j - 1]
        yield a, x


def test_rn32_matches_numpy_float32():
    np = pytest.importorskip("numpy")
    rng = synth.Rng(11, 1)
    vals = list(rng.uniform(400, -1, 1) * 2.0 ** rng.uniform(400, -140, 120))
    vals += [1 + 2 ** -24, 1 + 3 * 2 ** -24, 2.0 ** -149 * 1.5, 2.0 ** -150]
    for v in vals:
        assert rn32(Q(v)) == Q(float(np.float32(v))), v


@pytest.mark.parametrize("seed", range(3))
def test_emulated_row_sum_meets_its_bound(seed):
    worst = Q(0)
    for a, x in rows(seed, 160):
        err, scale = row_error(a, x)
        assert err <= bound(len(a), scale), (len(a), float(err / scale))
        worst = max(worst, err / bound(len(a), scale))
    assert worst < 1


def test_bound_is_below_the_fp64_tolerance():
    assert float(bound(48, 1)) < 9.6e-13 < 1e-12


def test_a_dropped_low_word_breaks_the_bound():
    broken = 0
    for a, x in rows(7, 40):
        err, scale = row_error(a, x, keep_low=False)
        broken += err > bound(len(a), scale)
    assert broken > 0
