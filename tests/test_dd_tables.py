"""Host check of the double-float difference-form tables (no GPU).

The residual update of a refinement step from zero evaluates L(d) = sum_i S_i d T_i^T
(Sec. 5, operator L~) in difference form in double-float arithmetic.  Its tables come
from the library's FP64 band tables (`mofem_host_tables`, pinned against the oracle's
assembly elsewhere); this test checks the transformation itself against exact rational
arithmetic:

* off the diagonal slot, (hi, lo) is the FP32 split of the FP64 coefficient;
* on it, the row sum of the FP64 coefficients (computed here exactly with Fractions),
  to one rounding of the pair, in every t-table and in the s-tables of the
  difference-form terms; the plain diagonal coefficient in the others;
* t-table 0 holds N = D^-1 (M_t - D) and D = rowsum M_t, so that D (1 + N) reproduces
  the mass row exactly up to that rounding, the exact mass split d M_t^T = D (d + d N^T).

A plausible mistake (a row sum left in FP64 rounding, a lost low part, N without the
division, a term put in the wrong form) fails one of these.
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_2109_01173_gb300.inputs import Profile, ZERO, SIN_TOP

TWO = (Profile(c2=0.1), Profile(c0=1.0, ca=0.2, cf=1.0))
U48 = 2.0 ** -47   # one rounding of a double-float pair, with slack for its two parts


def _split(c):
    hi = np.float32(c)
    lo = np.float32(c - float(hi))
    return hi, lo


@pytest.fixture(scope="module")
def mf():
    import paper_2109_01173_gb300.mofem as m
    return m


@pytest.mark.parametrize("k,n,dom,bc", [(2, 65, "one", 0), (1, 41, "two", 1), (0, 33, "one", 0),
                                        (3, 31, "two", 0), (4, 33, "one", 1), (2, 33, "two", 0)])
def test_dd_tables(mf, k, n, dom, bc):
    g1, g2 = (ZERO, SIN_TOP) if dom == "one" else TWO
    t = mf.host_dd_tables(g1, g2, k, n, 1.5, bc=bc)
    base = t["base"]
    S, T, K, nt, q = base["S"], base["T"], base["K"], base["n_terms"], base["q"]
    P = 2 * K + 1
    assert nt == (5 if dom == "one" else 8)
    dmask = 0x19 if nt == 5 else 0xF1
    for table, hi, lo, kind in ((T, t["T_hi"], t["T_lo"], "T"), (S, t["S_hi"], t["S_lo"], "S")):
        for i in range(nt):
            diff = kind == "T" or (dmask >> i) & 1
            for r in range(q):
                row = [float(table[i][j][r]) for j in range(P)]
                exact_rs = sum((Fraction(c) for c in row), Fraction(0))
                scale = max(abs(c) for c in row) or 1.0
                mass_split = kind == "T" and i == 0
                for j in range(P):
                    h, l = hi[i][j][r], lo[i][j][r]
                    if j == K and diff:
                        got = Fraction(float(h)) + Fraction(float(l))
                        assert abs(got - exact_rs) <= U48 * abs(exact_rs) + 2.0 ** -100 * scale, (kind, i, r)
                    elif j != K and mass_split:
                        # N_j = T0_j / D with D the exact row sum: D N_j reproduces T0_j
                        if exact_rs != 0:
                            nj = Fraction(float(h)) + Fraction(float(l))
                            assert abs(nj * exact_rs - Fraction(row[j])) <= U48 * abs(row[j]) + 2.0 ** -100 * scale, (i, r, j)
                    else:
                        eh, el = _split(row[j])
                        assert h == eh and l == el, (kind, i, r, j)


def test_dd_tables_stiffness_row_sums(mf):
    """The interior rows of a stiffness factor sum to zero in exact arithmetic; the
    table's row sum is that of the FP64 coefficients (tiny, not the FP64-rounded sum of
    them, which would be a rounding error ~1e-16 of the coefficients)."""
    t = mf.host_dd_tables(ZERO, SIN_TOP, 2, 65, 1.0)
    base = t["base"]
    K, q = base["K"], base["q"]
    T = base["T"]
    # T table 1 is K_t (stiffness, t-factor): interior rows have (near) zero row sums
    for r in range(K, q - K):
        row = [float(T[1][j][r]) for j in range(2 * K + 1)]
        exact = sum((Fraction(c) for c in row), Fraction(0))
        got = Fraction(float(t["T_hi"][1][K][r])) + Fraction(float(t["T_lo"][1][K][r]))
        assert abs(got - exact) <= U48 * abs(exact) + 2.0 ** -100, r
        assert abs(float(exact)) <= 1e-13 * max(abs(c) for c in row)
