"""Model of the fold of the refinement's step from zero (CPU, no GPU).

The fold forms the step d = hi + lo (+ alpha Q) in double-float arithmetic and rounds the
low part onto the FP64 grid of the high part (multiples of 2^(e_hi - 52)), so that the
FP64 iterate can be set to hi + lo exactly: the residual update then subtracts L of
exactly the step the iterate took.  This models that arithmetic with numpy FP32
operations and checks, on random and unnormalised pairs (and products alpha q pending),
that (double) hi + (double) lo equals the exact sum of the pair, and that the step
differs from the FP64-formed step by no more than a few roundings of 2^-48 of its
operands.
"""
from fractions import Fraction

import numpy as np

f32 = np.float32


def _two_sum(a, b):
    s = f32(a + b)
    v = f32(s - a)
    return s, f32(f32(a - f32(s - v)) + f32(b - v))


def _fma(a, b, c):
    # fl32(a * b + c): the product is exact in FP64; the FP64 sum then rounds at 2^-53
    return f32(float(a) * float(b) + float(c))


def _fold_zero(h, l, aph, apl, q, pend):
    s, lo = _two_sum(h, l)
    if pend:
        p = f32(aph * q)
        e = _fma(aph, q, -p)
        e = _fma(apl, q, e)
        t, r = _two_sum(s, p)
        s, lo = t, f32(f32(lo + e) + r)
    H, L = _two_sum(s, lo)
    if H != 0:
        eh = int(np.frexp(H)[1]) - 1          # exponent of H (H = m 2^eh, 1 <= |m| < 2)
        L = f32(np.ldexp(np.rint(np.ldexp(L, 52 - eh)), eh - 52)) if eh >= -97 else f32(0.0)
    return H, L


def test_fold_from_zero_is_exact():
    rng = np.random.default_rng(11)
    worst = 0.0
    for _ in range(20000):
        sc = int(rng.integers(-40, 40))
        d = np.ldexp(rng.uniform(-1, 1), sc)
        h = f32(d)
        l = f32(d - float(h))
        if rng.integers(4) == 0:                   # unnormalised low part
            l = f32(np.ldexp(rng.uniform(-1, 1), sc - 20 - int(rng.integers(30))))
        if rng.integers(40) == 0:
            h = f32(0.0)
        ap = np.ldexp(rng.uniform(-1, 1), int(rng.integers(-20, 20)))
        aph = f32(ap)
        apl = f32(ap - float(aph))
        q = f32(np.ldexp(rng.uniform(-1, 1), sc + int(rng.integers(-8, 8))))
        pend = bool(rng.integers(2))
        H, L = _fold_zero(h, l, aph, apl, q, pend)
        u = float(H) + float(L)                   # the iterate after the fold (FP64)
        assert Fraction(u) == Fraction(float(H)) + Fraction(float(L))
        want = Fraction(float(h)) + Fraction(float(l))
        mag = max(abs(float(h) + float(l)), 0.0)
        if pend:
            want += Fraction(ap) * Fraction(float(q))
            mag = max(mag, abs(ap * float(q)))
        if mag > 2.0 ** -90:
            worst = max(worst, float(abs(Fraction(u) - want)) / mag)
    assert worst <= 2.0 ** -44, worst
