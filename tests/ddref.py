"""Double-double reference evaluation of the multiterm operator for tests.

B - sum_i S_i U T_i^T (or the sum alone) on band tables S, T [term][slot][row], slot j
of row r holding the coefficient of column r + j - K, in double-double arithmetic:
every product exact (Dekker's product with Veltkamp's split, no FMA needed), every sum
carried with its rounding error.  Far more accurate than an FP64 evaluation, whose
rounding of the t-pass product the s-stiffness amplifies.  Test infrastructure only.
"""
import numpy as np


def two_prod(a, b):
    """a * b = p + e exactly."""
    def split(x):
        c = 134217729.0 * x
        hi = c - (c - x)
        return hi, x - hi
    p = a * b
    ah, al = split(a)
    bh, bl = split(b)
    return p, ((ah * bh - p) + ah * bl + al * bh) + al * bl


def two_sum(a, b):
    """a + b = s + r exactly."""
    s = a + b
    v = s - a
    return s, (a - (s - v)) + (b - v)


def shift(X, off, axis):
    """Y[.., i] = X[.., i + off] along axis (0 or 1 of a 2D array), zero outside."""
    Y = np.zeros_like(X)
    n = X.shape[axis]
    src = [slice(None)] * 2
    dst = [slice(None)] * 2
    if off >= 0:
        src[axis], dst[axis] = slice(off, n), slice(0, n - off)
    else:
        src[axis], dst[axis] = slice(0, n + off), slice(-off, n)
    Y[tuple(dst)] = X[tuple(src)]
    return Y


def apply_dd(S, T, K, U):
    """sum_i S_i U T_i^T as a double-double pair (hi, lo)."""
    P = 2 * K + 1
    yh = np.zeros_like(U)
    yl = np.zeros_like(U)
    for i in range(S.shape[0]):
        vh = np.zeros_like(U)
        vl = np.zeros_like(U)
        for l in range(P):
            p, e = two_prod(T[i][l][None, :], shift(U, l - K, 1))
            vh, t = two_sum(vh, p)
            vl = vl + (t + e)
        vh, vl = two_sum(vh, vl)
        for j in range(P):
            c = S[i][j][:, None]
            p, e = two_prod(c, shift(vh, j - K, 0))
            yh, t = two_sum(yh, p)
            yl = yl + (t + e + c * shift(vl, j - K, 0))
    return yh, yl


def residual_dd(S, T, K, B, U):
    """B - sum_i S_i U T_i^T, rounded once to FP64."""
    yh, yl = apply_dd(S, T, K, U)
    r, t = two_sum(B, -yh)
    return r + (t - yl)
