"""The reduced-precision bound for rows whose CSR remainder is summed in FP64.

FP32 / BF16 products accumulate in FP32, except a remainder row (Fig. 13,
first loop) longer than oracle.REM_LONG entries: it is summed in FP64 and
rounded once into the FP32 accumulator.  These tests pin the oracle's bound
for that arithmetic to exact rational arithmetic (every rounding simulated
exactly with fractions), show that it is sharp enough to reject a product
that ignored the rule, and pin oracle.long_remainder."""
from fractions import Fraction

import numpy as np

import oracle
import synth


def _nearest(q: Fraction, cands) -> Fraction:
    """Round-to-nearest-even choice of q among neighbouring floats."""
    best = None
    for c in cands:
        d = abs(Fraction(float(c)) - q)
        odd = int(np.asarray(c).view(np.uint32 if c.dtype == np.float32 else np.uint64)) & 1
        if best is None or (d, odd) < best[0]:
            best = ((d, odd), c)
    return Fraction(float(best[1]))


def fl32(q: Fraction) -> Fraction:
    f = np.float32(float(q))  # within one ulp of the correctly rounded value
    return _nearest(q, (np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))))


def fl64(q: Fraction) -> Fraction:
    return Fraction(float(q))  # int / int true division rounds correctly


def row_fp32_kernel(rem, diag):
    """One row as the kernels compute it for an FP32 handle: the remainder
    in column order (FP64 sum rounded once if longer than REM_LONG, else FP32
    FMAs from zero), then the diagonal terms as FP32 FMAs."""
    if len(rem) > oracle.REM_LONG:
        s = Fraction(0)
        for a, x in rem:
            s = fl64(a * x + s)
        acc = fl32(s)
    else:
        acc = Fraction(0)
        for a, x in rem:
            acc = fl32(a * x + acc)
    for a, x in diag:
        acc = fl32(a * x + acc)
    return acc


def row_fp32_only(rem, diag):
    acc = Fraction(0)
    for a, x in list(rem) + list(diag):
        acc = fl32(a * x + acc)
    return acc


def _f32_terms(rng, k):
    mag = 10.0 ** rng.uniform(k, -3, 3)
    sgn = np.where(rng.uniform(k, 0, 1) < 0.5, -1.0, 1.0)
    a = oracle.round_f32(sgn * mag)
    x = oracle.round_f32(rng.uniform(k, -1, 1))
    return [(Fraction(float(ai)), Fraction(float(xi))) for ai, xi in zip(a, x)]


def test_long_row_bound_holds_in_exact_arithmetic():
    rng = synth.Rng(11, 4)
    for L in (1, 64, 65, 200, 1500):
        for kd in (0, 3, 27):
            for _ in range(2):
                rem, diag = _f32_terms(rng, L), _f32_terms(rng, kd)
                exact = sum(a * x for a, x in rem + diag)
                absrow = float(sum(abs(a * x) for a, x in rem + diag))
                got = row_fp32_kernel(rem, diag)
                lr = L if L > oracle.REM_LONG else 0
                b = oracle.bound_vs_stored(absrow, L + kd, "f32", lr)
                assert float(abs(got - exact)) <= b, (L, kd)
                # the bound without the rule is looser, never tighter
                assert b <= oracle.bound_vs_stored(absrow, L + kd, "f32")


def test_long_row_bound_rejects_fp32_accumulation():
    # 2^25 then ones: in FP32 every +1 is lost (ulp(2^25) = 4, ties to even),
    # in FP64 none is.  With 64 ones the FP32-only result misses by 64, more
    # than the bound for the FP64 remainder allows; the kernel's arithmetic
    # is exact here.
    big = Fraction(2 ** 25)
    for ones in (64, 300):
        rem = [(big, Fraction(1))] + [(Fraction(1), Fraction(1))] * ones
        diag = [(Fraction(4), Fraction(1)), (Fraction(8), Fraction(1)), (Fraction(4), Fraction(1))]
        exact = big + ones + 16
        assert row_fp32_kernel(rem, diag) == exact
        assert row_fp32_only(rem, diag) == big + 16
        L = ones + 1
        b = oracle.bound_vs_stored(float(exact), L + 3, "f32", L)
        assert b < ones                      # a product ignoring the rule fails
        assert oracle.bound_vs_stored(float(exact), L + 3, "f32") >= ones  # the loose bound would not
    # 63 ones (remainder of 64 entries, not long): FP32 accumulation by rule
    rem = [(big, Fraction(1))] + [(Fraction(1), Fraction(1))] * 63
    assert row_fp32_kernel(rem, []) == big
    assert abs(float(big + 63 - big)) <= oracle.bound_vs_stored(float(big + 63), 64, "f32", 0)


def test_long_remainder_rows_of_a_converted_matrix():
    n = 400
    d = np.zeros((n, n))
    d[np.arange(n), np.arange(n)] = 2.0
    d[10, 100:164] = 1.0        # 64 off-band entries: not long
    d[20, 100:165] = 1.0        # 65: long
    d[399, 0:300] = 0.5         # 300: long (last row)
    A = synth.from_dense(d)
    for dt in ("f32", "bf16"):
        M = oracle.convert(A, 128, 0.6, dt)
        lr = oracle.long_remainder(M)
        want = np.zeros(n, dtype=np.int64)
        want[20], want[399] = 65, 300
        assert np.array_equal(lr, want), dt
    assert not np.any(oracle.long_remainder(oracle.convert(A, 128, 0.6, "f64")))
