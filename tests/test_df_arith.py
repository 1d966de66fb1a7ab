"""The double-float method of SS_MODE_DF, checked on the CPU in exact rational
arithmetic: a float32 emulation (numpy float32 operations, round-to-nearest)
of the operand split, the TwoProduct / TwoSum multiply-subtract and the
normalised product, against the bounds the library documents (about 48
significant bits per operand, 2^-47 relative split error).  This checks the
method; the CUDA kernels themselves are checked against the oracle by the GPU
parity tests."""
from fractions import Fraction

import numpy as np
import pytest

F32 = np.float32


def trunc_bits(x: float, keep: int) -> float:
    """x with its significand truncated to `keep` bits (float64 in, exact)."""
    if x == 0.0 or not np.isfinite(x):
        return x
    m, e = np.frexp(x)                      # x = m * 2^e, 0.5 <= |m| < 1
    scale = float(2 ** keep)
    return float(np.ldexp(np.trunc(m * scale) / scale, e))


TINY = 2.0 ** -126                          # smallest normal float32


def split(x: float):
    """hi = the leading 24 significant bits of x, lo = the next 24 (both
    truncated), as the integer split of the kernels does; a lo below the
    float32 normal range is flushed to zero, as there."""
    hi = trunc_bits(x, 24)
    lo = trunc_bits(x - hi, 24)             # x - hi is exact in float64
    if abs(lo) < TINY:
        lo = 0.0
    return F32(hi), F32(lo)


def fma32(a, b, c):
    # a*b is exact in float64 (48 bits); the error terms below are exact
    # sums, so one float64 rounding then one float32 rounding is the FMA's.
    return F32(float(a) * float(b) + float(c))


def df_msub(ah, al, xh, xl, yh, yl):
    """(ah, al) -= (xh + xl) (yh + yl), the kernels' sequence of operations."""
    p = F32(xh * yh)
    pe = fma32(xh, yh, -p)
    pe = F32(pe + fma32(xh, yl, F32(xl * yh)))
    s = F32(ah - p)
    bb = F32(s - ah)
    err = F32(F32(ah - F32(s - bb)) + F32(-p - bb))
    return s, F32(al + F32(err - pe))


def df_mul(vh, vl, rh, rl):
    p = F32(vh * rh)
    e = fma32(vh, rh, -p)
    e = fma32(vh, rl, e)
    e = fma32(vl, rh, e)
    s = F32(p + e)
    return s, F32(e - F32(s - p))


def exact(*vals):
    return sum((Fraction(float(v)) for v in vals), Fraction(0))


@pytest.mark.parametrize("seed", range(5))
def test_split_keeps_48_bits(seed):
    # A low part that would be subnormal is flushed.  For |x| >= 2^-79 such a
    # low part is below 2^-126 <= 2^-47 |x|, so the 2^-47 bound holds (up to
    # the float32 overflow); between 2^-126 and 2^-79 only the 24 bits of the
    # high part are guaranteed.
    rng = np.random.default_rng(seed)
    for x in rng.standard_normal(2000) * 10.0 ** rng.uniform(-37, 37, 2000):
        x = float(x)
        if abs(x) < TINY:
            continue                        # outside the documented range
        hi, lo = split(x)
        assert float(hi) == trunc_bits(x, 24)
        err = abs(Fraction(x) - exact(hi, lo))
        if abs(x) >= 2.0 ** -79:
            assert err <= Fraction(2) ** -47 * abs(Fraction(x))
        elif abs(x) >= TINY:
            assert err <= Fraction(2) ** -23 * abs(Fraction(x))


@pytest.mark.parametrize("n", [1, 16, 128, 512])
def test_dot_product_error_bound(n):
    # T = c - sum a_i b_i accumulated term by term as the block updates do.
    rng = np.random.default_rng(n)
    a, b = rng.standard_normal(n), rng.standard_normal(n)
    c = float(rng.standard_normal())
    ah, al = split(c)
    for x, y in zip(a, b):
        xh, xl = split(float(x))
        yh, yl = split(float(y))
        ah, al = df_msub(ah, al, xh, xl, yh, yl)
    ref = Fraction(c) - sum((Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b)), Fraction(0))
    scale = abs(Fraction(c)) + sum((abs(Fraction(float(x)) * Fraction(float(y))) for x, y in zip(a, b)), Fraction(0))
    err = abs(exact(ah, al) - ref)
    # Splits: 3 x 2^-47 per term; each update's rounding of the low part
    # contributes about 2^-48 of the running magnitude.
    assert err <= (n + 2) * Fraction(2) ** -45 * scale
    # And it is far more accurate than the FP32 dot product.
    f32 = F32(c)
    for x, y in zip(a, b):
        f32 = F32(f32 - F32(F32(x) * F32(y)))
    if n >= 16:
        assert err * 1000 < abs(Fraction(float(f32)) - ref) + Fraction(2) ** -60 * scale


def test_normalised_product():
    rng = np.random.default_rng(7)
    for _ in range(2000):
        v, r = rng.standard_normal(2) * 10.0 ** rng.uniform(-10, 10, 2)
        vh, vl = split(float(v))
        rh, rl = split(float(r))
        xh, xl = df_mul(vh, vl, rh, rl)
        exact_prod = exact(vh, vl) * exact(rh, rl)
        assert abs(exact(xh, xl) - exact_prod) <= Fraction(2) ** -44 * abs(exact_prod)
        assert abs(float(xl)) <= abs(float(xh)) * 2.0 ** -23         # normalised
