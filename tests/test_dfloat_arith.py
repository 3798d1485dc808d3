"""The double-float arithmetic of the FSIM_DFLOAT kernels, step by step in NumPy float32.

The kernels (csrc/dfloat.cuh, csrc/boys.cuh) keep a value as hi + lo, two FP32
numbers, and build every operation from error-free transformations: Knuth's
two-sum, Dekker's fast two-sum, and the exact product p + e = a b with
e = fma(a, b, -p).  Here the same steps run on float32 scalars (round to
nearest, like the _rn intrinsics; an FP32 fused multiply-add is emulated in
float64, where a product of two float32 values is exact) and are checked
against exact rational arithmetic and float64, to the error bounds the
kernels rely on:
  * two-sum and the exact product are exact;
  * multiply, multiply-add: relative error a few 2^-47 of the operands' scale;
  * 1/sqrt(x) from a 2-ulp FP32 estimate and one Newton step: below 2^-41;
  * e^x on |x| <= 1/32 by its Taylor series to x^7: below 2^-47 (the
    truncation is below 2^-55; the rest is double-float rounding).
The GPU parity tests check the kernels' results against the oracle; these
pin the arithmetic they are built from.
"""
import math
from fractions import Fraction

import numpy as np

f32 = np.float32


def fadd(a, b):
    return f32(f32(a) + f32(b))


def fsub(a, b):
    return f32(f32(a) - f32(b))


def fmul(a, b):
    return f32(f32(a) * f32(b))


def ffma(a, b, c):
    # exact product in float64, one rounding to float32 (the sum in float64 is exact
    # for the operands used here up to 2^-70 relative, far below what is tested)
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def split(d):
    hi = f32(d)
    return hi, f32(np.float64(d) - np.float64(hi))


def value(x):
    return Fraction(float(x[0])) + Fraction(float(x[1]))


def fast_two_sum(s, e):
    h = fadd(s, e)
    return h, fsub(e, fsub(h, s))


def add(x, y):
    s = fadd(x[0], y[0])
    v = fsub(s, x[0])
    e = fadd(fsub(x[0], fsub(s, v)), fsub(y[0], v))
    e = fadd(e, fadd(x[1], y[1]))
    return fast_two_sum(s, e)


def mul(x, y):
    p = fmul(x[0], y[0])
    e = ffma(x[0], y[0], -p)
    e = ffma(x[0], y[1], e)
    e = ffma(x[1], y[0], e)
    return fast_two_sum(p, e)


def fma(x, y, z):
    p = fmul(x[0], y[0])
    e = ffma(x[0], y[0], -p)
    e = ffma(x[0], y[1], e)
    e = ffma(x[1], y[0], e)
    s = fadd(p, z[0])
    v = fsub(s, p)
    f = fadd(fsub(p, fsub(s, v)), fsub(z[0], v))
    f = fadd(f, fadd(e, z[1]))
    return fast_two_sum(s, f)


def rsqrt(x, r):
    """One Newton step from the FP32 estimate r of 1/sqrt(x.hi)."""
    rr = fmul(r, r)
    r2 = (rr, ffma(r, r, -rr))
    xr2 = mul(x, r2)
    e = fsub(fsub(f32(1.0), xr2[0]), xr2[1])
    return fast_two_sum(r, fmul(fmul(f32(0.5), r), e))


def rand_doubles(rng, n, lo=-3.0, hi=3.0):
    return rng.uniform(-1, 1, n) * 10.0 ** rng.uniform(lo, hi, n)


def test_two_sum_and_product_are_exact():
    rng = np.random.default_rng(0)
    for a, b in zip(rand_doubles(rng, 2000, -8, 8), rand_doubles(rng, 2000, -8, 8)):
        a, b = f32(a), f32(b)
        s = fadd(a, b)
        v = fsub(s, a)
        e = fadd(fsub(a, fsub(s, v)), fsub(b, v))
        assert Fraction(float(s)) + Fraction(float(e)) == Fraction(float(a)) + Fraction(float(b))
        p = fmul(a, b)
        q = ffma(a, b, -p)
        assert Fraction(float(p)) + Fraction(float(q)) == Fraction(float(a)) * Fraction(float(b))


def test_split_keeps_48_bits():
    rng = np.random.default_rng(1)
    for d in rand_doubles(rng, 2000, -20, 20):
        x = split(d)
        assert abs(value(x) - Fraction(float(d))) <= abs(Fraction(float(d))) * Fraction(1, 2 ** 48)


def test_mul_and_fma_error_bounds():
    rng = np.random.default_rng(2)
    n = 3000
    X, Y, Z = rand_doubles(rng, n), rand_doubles(rng, n), rand_doubles(rng, n)
    worst_mul = worst_fma = 0.0
    for a, b, c in zip(X, Y, Z):
        x, y, z = split(a), split(b), split(c)
        exact = value(x) * value(y)
        got = value(mul(x, y))
        worst_mul = max(worst_mul, float(abs(got - exact) / abs(exact)))
        exact = value(x) * value(y) + value(z)
        scale = abs(value(x) * value(y)) + abs(value(z))
        got = value(fma(x, y, z))
        worst_fma = max(worst_fma, float(abs(got - exact) / scale))
    assert worst_mul < 4 * 2.0 ** -47, worst_mul
    assert worst_fma < 4 * 2.0 ** -47, worst_fma


def test_cancelling_sum_error_is_relative_to_the_operands():
    # x + y with x ~ -y: the error is bounded by the operands' size, not by |x + y|
    rng = np.random.default_rng(3)
    for a in rand_doubles(rng, 2000):
        b = -a * (1.0 + rng.uniform(-1e-6, 1e-6))
        x, y = split(a), split(b)
        got = value(add(x, y))
        exact = value(x) + value(y)
        assert abs(got - exact) <= (abs(value(x)) + abs(value(y))) * Fraction(4, 2 ** 47)


def test_newton_rsqrt():
    rng = np.random.default_rng(4)
    worst = 0.0
    for s in 10.0 ** rng.uniform(-1, 4, 2000):
        x = split(s)
        # an FP32 estimate off by up to 2 ulp, as a hardware approximation may be
        r0 = f32(1.0 / math.sqrt(float(x[0])))
        r0 = np.nextafter(r0, f32(np.inf) if rng.random() < 0.5 else f32(0), dtype=np.float32)
        r0 = np.nextafter(r0, f32(np.inf) if rng.random() < 0.5 else f32(0), dtype=np.float32)
        got = float(value(rsqrt(x, r0)))
        ref = 1.0 / math.sqrt(float(value(x)))
        worst = max(worst, abs(got - ref) / ref)
    assert worst < 2.0 ** -41, worst


def test_exp_taylor_on_the_grid_interval():
    # e^x = sum_{k <= 7} x^k / k! by Horner in double-float, |x| <= 1/32 (the Boys grid)
    inv_fact = [split(1.0 / math.factorial(k)) for k in range(8)]
    worst = 0.0
    for xv in np.linspace(-1.0 / 32, 1.0 / 32, 257):
        x = split(xv)
        ex = inv_fact[7]
        for k in range(6, -1, -1):
            ex = fma(ex, x, inv_fact[k])
        ref = math.exp(float(value(x)))
        worst = max(worst, abs(float(value(ex)) - ref) / ref)
    assert worst < 2.0 ** -47, worst
