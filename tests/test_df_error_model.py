"""Error model of the refinement's double-float residual evaluation (CPU, no GPU).

A numpy model of the arithmetic of the two double-float forms of L(d) = sum_i S_i d T_i^T
(Sec. 5, operator L~): FP32 operations only, error-free transforms for products and sums,
on the library's own tables (`mofem_host_tables`, `mofem_host_dd_tables`), for a smooth
step d of the size of U (the first refinement step from zero).  Measured against a
double-double evaluation on the same FP64 coefficients, relative to ||L(d)||:

* the plain form's error grows like q^2 (a rounding of the t-pass mass product is
  second-differenced by the s-stiffness) and is far above the FP64 evaluation noise;
* the difference form with exact row sums, exact input differences and the exact mass
  split of term 0 grows like q and stays below the FP64 difference form's error.

These are the figures on which the step from zero was moved from an FP64 recomputation
to the double-float difference form.  The model follows the kernels' order of operations
but not their register layout; it checks the method, the GPU tests check the kernels.
"""
import numpy as np
import pytest

from paper_2109_01173_gb300.inputs import ZERO, SIN_TOP
from ddref import apply_dd, shift as _shift

f32 = np.float32


# ---- FP32 error-free transforms (numpy float32 rounds each operation once) ----------
def _two_sum(a, b):
    s = (a + b).astype(f32)
    v = (s - a).astype(f32)
    return s, ((a - (s - v)) + (b - v)).astype(f32)


def _prod(ah, al, bh, bl):
    """(ah + al)(bh + bl): the high product and its exact error plus the cross terms."""
    p = (ah * bh).astype(f32)
    e = (ah.astype(np.float64) * bh - p).astype(f32)          # exact: the product's rounding error
    e = (ah.astype(np.float64) * bl + e).astype(f32)
    e = (al.astype(np.float64) * bh + e).astype(f32)
    return p, e


class _DF:
    def __init__(self, h, l):
        self.h, self.l = h, l

    def renorm(self):
        h = (self.h + self.l).astype(f32)
        return _DF(h, (self.l - (h - self.h)).astype(f32))


def _chain(pairs):
    """Sum of products, high part carried, every rounding error collected in the low part."""
    out = None
    for (ah, al), x in pairs:
        p, e = _prod(ah, al, x.h, x.l)
        if out is None:
            out = _DF(p, e)
        else:
            t, r = _two_sum(out.h, p)
            out = _DF(t, (out.l + (r + e).astype(f32)).astype(f32))
    return out


def _sub_exact(x, c):
    s1, r1 = _two_sum(x.h, -c.h)
    s2, r2 = _two_sum(x.l, -c.l)
    t, e1 = _two_sum(s1, s2)
    lo = ((e1 + r1).astype(f32) + r2).astype(f32)
    h = (t + lo).astype(f32)
    return _DF(h, (lo - (h - t)).astype(f32))


def _sub_df(x, c):
    s, r = _two_sum(x.h, -c.h)
    lo = ((x.l - c.l).astype(f32) + r).astype(f32)
    h, l = _two_sum(s, lo)
    return _DF(h, l)


def _sh(x, off, axis):
    return _DF(_shift(x.h, off, axis), _shift(x.l, off, axis))


def _plain_df(S, T, K, x):
    P = 2 * K + 1
    split = lambda v: (v.astype(f32), (v - v.astype(f32).astype(np.float64)).astype(f32))
    y = None
    for i in range(S.shape[0]):
        th = [split(T[i][l]) for l in range(P)]
        V = _chain([((h[None, :], l[None, :]), _sh(x, l_ - K, 1)) for l_, (h, l) in enumerate(th)]).renorm()
        sh = [split(S[i][j]) for j in range(P)]
        W = _chain([((h[:, None], l[:, None]), _sh(V, j - K, 0)) for j, (h, l) in enumerate(sh)])
        y = W if y is None else _acc(y, W)
    return y.h.astype(np.float64) + y.l.astype(np.float64)


def _acc(y, w):
    t, r = _two_sum(y.h, w.h)
    return _DF(t, (y.l + (r + w.l).astype(f32)).astype(f32))


def _diff_df(dd, K, x, nt):
    """The difference form of the step from zero, on the library's double-float tables."""
    P = 2 * K + 1
    dm = 0x19 if nt == 5 else 0xF1
    Sh, Sl, Th, Tl = dd["S_hi"], dd["S_lo"], dd["T_hi"], dd["T_lo"]
    dx = {l: _sub_exact(_sh(x, l - K, 1), x) for l in range(P) if l != K}
    rings = []
    for i in range(nt):
        pairs = [] if i == 0 else [((Th[i][K][None, :], Tl[i][K][None, :]), x)]
        pairs += [((Th[i][l][None, :], Tl[i][l][None, :]), dx[l]) for l in range(P) if l != K]
        rings.append(_chain(pairs).renorm())

    def spass(i, V, exact):
        c = lambda j: (Sh[i][j][:, None], Sl[i][j][:, None])
        if (dm >> i) & 1:
            sub = _sub_exact if exact else _sub_df
            pairs = [(c(K), V)] + [(c(j), sub(_sh(V, j - K, 0), V)) for j in range(P) if j != K]
        else:
            pairs = [(c(j), _sh(V, j - K, 0)) for j in range(P)]
        return _chain(pairs)

    ya, yb = spass(0, x, True).renorm(), spass(0, rings[0], False).renorm()
    s, r = _two_sum(ya.h, yb.h)
    sab = _DF(s, ((r + ya.l).astype(f32) + yb.l).astype(f32)).renorm()
    y = _chain([((Th[0][K][None, :] + 0 * sab.h, Tl[0][K][None, :] + 0 * sab.h), sab)])
    for i in range(1, nt):
        y = _acc(y, spass(i, rings[i], False).renorm())
    return y.h.astype(np.float64) + y.l.astype(np.float64)


def _diff_fp64(S, T, K, x):
    """The FP64 difference form (row sums in FP64, t-pass first, no mass split)."""
    P = 2 * K + 1
    nt = S.shape[0]
    dm = 0x19 if nt == 5 else 0xF1
    y = np.zeros_like(x)
    for i in range(nt):
        V = T[i].sum(axis=0)[None, :] * x
        for l in range(P):
            if l != K:
                V = V + T[i][l][None, :] * (_shift(x, l - K, 1) - x)
        if (dm >> i) & 1:
            W = S[i].sum(axis=0)[:, None] * V
            for j in range(P):
                if j != K:
                    W = W + S[i][j][:, None] * (_shift(V, j - K, 0) - V)
        else:
            W = sum(S[i][j][:, None] * _shift(V, j - K, 0) for j in range(P))
        y = y + W
    return y


def _errors(mf, n):
    tb = mf.host_tables(ZERO, SIN_TOP, 2, n, 1.0)
    dd = mf.host_dd_tables(ZERO, SIN_TOP, 2, n, 1.0)
    S, T, K, q, nt = tb["S"], tb["T"], tb["K"], tb["q"], tb["n_terms"]
    rng = np.random.default_rng(1)
    s = np.linspace(0.0, 1.0, n)[1:-1]
    d = np.zeros((q, q))
    for a in range(1, 7):
        for b in range(1, 7):
            d += rng.standard_normal() / (a * a + b * b) ** 2 * np.outer(np.sin(a * np.pi * s), np.sin(b * np.pi * s))
    xh = d.astype(f32)
    xl = (d - xh.astype(np.float64)).astype(f32)
    x64 = xh.astype(np.float64) + xl.astype(np.float64)     # the step exactly
    rh, rl = apply_dd(S, T, K, x64)
    nrm = np.linalg.norm(rh)
    err = lambda y: np.linalg.norm((y - rh) - rl) / nrm
    x = _DF(xh, xl)
    return dict(q=q, plain=err(_plain_df(S, T, K, x)), diff=err(_diff_df(dd, K, x, nt)),
                fp64=err(_diff_fp64(S, T, K, x64)))


@pytest.fixture(scope="module")
def mf():
    import paper_2109_01173_gb300.mofem as m
    return m


@pytest.fixture(scope="module")
def errs(mf):
    return [_errors(mf, n) for n in (129, 257)]


def test_plain_double_float_grows_like_q_squared(errs):
    a, b = errs
    assert b["plain"] / a["plain"] > 3.0, (a, b)
    assert b["plain"] > 10 * b["fp64"], b


def test_difference_form_grows_like_q_and_beats_fp64(errs):
    a, b = errs
    assert b["diff"] / a["diff"] < 2.6, (a, b)
    assert b["diff"] < b["fp64"], b
    assert b["diff"] < 2.0 ** -48 * 8 * b["q"], b
