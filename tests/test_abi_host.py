"""CPU-only checks of libmofem: it loads, exports every entry point that
include/mofem.h declares, validates arguments, and its host-side setup tables
(C++ assembly, written independently of the oracle) equal the oracle's 1D
factor matrices for every degree, both boundary conditions and both the
five-term and eight-term operators."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle.operator import Problem
from paper_2109_01173_gb300.inputs import Profile, ZERO, SIN_TOP

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mofem():
    from paper_2109_01173_gb300 import build
    build.build()
    import paper_2109_01173_gb300.mofem as m
    return m


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(mofem_\w+)\s*\(", src)
    return sorted(set(names))


def test_exports_every_declared_symbol(mofem):
    lib = ctypes.CDLL(mofem.LIB_PATH)
    decl = declared_functions()
    assert len(decl) >= 10
    for name in decl:
        assert hasattr(lib, name), name


def test_status_strings(mofem):
    assert mofem.LIB.mofem_status_string(0) == b"MOFEM_OK"
    assert mofem.LIB.mofem_status_string(6) == b"MOFEM_ERR_NOT_CONVERGED"


def test_invalid_arguments_rejected_without_gpu(mofem):
    p, keep = mofem.make_profile(ZERO)
    p2, keep2 = mofem.make_profile(SIN_TOP)
    h = ctypes.c_void_p()
    L = mofem.LIB
    # k out of range, (n-1) not divisible by k, Neumann with gamma = 0, null handle out
    assert L.mofem_setup(ctypes.byref(p), ctypes.byref(p2), 5, 65, 1.0, 0, None, None, ctypes.byref(h)) == 1
    assert L.mofem_setup(ctypes.byref(p), ctypes.byref(p2), 3, 65, 1.0, 0, None, None, ctypes.byref(h)) == 1
    assert L.mofem_setup(ctypes.byref(p), ctypes.byref(p2), 2, 65, 0.0, 1, None, None, ctypes.byref(h)) == 1
    assert L.mofem_setup(ctypes.byref(p), ctypes.byref(p2), 2, 65, 1.0, 0, None, None, None) == 1
    # non-positive height h = g2 - g1 is reported by the host tables without touching the GPU
    with pytest.raises(mofem.MofemError):
        mofem.host_tables(SIN_TOP, ZERO, 2, 9, 1.0)
    # the double-float difference-form tables: same argument checks
    assert L.mofem_host_dd_tables(ctypes.byref(p), ctypes.byref(p2), 5, 65, 1.0, 0, None, None, None) == 1
    assert L.mofem_host_dd_tables(ctypes.byref(p), ctypes.byref(p2), 3, 65, 1.0, 0, None, None, None) == 1
    assert L.mofem_host_dd_tables(None, ctypes.byref(p2), 2, 65, 1.0, 0, None, None, None) == 1
    with pytest.raises(mofem.MofemError):
        mofem.host_dd_tables(SIN_TOP, ZERO, 2, 9, 1.0)
    assert L.mofem_apply(None, None, None, 0, 0, None) == 1
    assert L.mofem_precond(None, None, None, 0, 0, None) == 1
    assert L.mofem_pcg_direction(None, None, None, None, None, None, None, 0, None, 0, None) == 1
    assert L.mofem_pcg_solve(None, None, None, 1e-10, 10, 0, None, None) == 1
    assert L.mofem_imex_step(None, 1.0, 1.0, None, None, None, 0, None, None) == 1
    assert L.mofem_imex_step_tol(None, 1.0, 1.0, None, None, None, 1e-10, 0, None, None) == 1
    assert L.mofem_imex_adjoint_step(None, 1.0, 1.0, None, None, None, None, None, 1e-10, 0, None, None) == 1
    assert L.mofem_rds_step(None, 1.0, None, None, None, 0.0, 0, None, None) == 1
    assert L.mofem_dib_kinetics(None, 1.0, None, None, None, None, 0, None) == 1
    assert L.mofem_dib_run(None, None, 1.0, 1.0, 1, None, 0.0, 0, None, None, None) == 1
    assert L.mofem_destroy(None) == 1
    assert L.mofem_get_eigen(None, None, None, None, None, None, None) == 1
    # the single-term stiffness preconditioners are singular under Neumann BC; the parabolic
    # one needs one positive gamma for the whole batch (its t-factor is shared)
    for pencil in (mofem.PENCIL_PRODUCT, mofem.PENCIL_AUA):
        o = mofem.make_opts(pencil=pencil)
        assert L.mofem_setup(ctypes.byref(p), ctypes.byref(p2), 2, 65, 1.0, 1, ctypes.byref(o), None,
                             ctypes.byref(h)) == 1
    o = mofem.make_opts(pencil=mofem.PENCIL_PARABOLIC)
    arr1, arr2 = (mofem.Profile * 2)(p, p), (mofem.Profile * 2)(p2, p2)
    gam = (ctypes.c_double * 2)(100.0, 50.0)
    assert L.mofem_setup_batched(2, arr1, arr2, 2, 65, gam, 0, ctypes.byref(o), None, ctypes.byref(h)) == 1
    assert L.mofem_setup(ctypes.byref(p), ctypes.byref(p2), 2, 65, 0.0, 0, ctypes.byref(o), None,
                         ctypes.byref(h)) == 1
    o = mofem.make_opts(pencil=5)
    assert L.mofem_setup(ctypes.byref(p), ctypes.byref(p2), 2, 65, 1.0, 0, ctypes.byref(o), None,
                         ctypes.byref(h)) == 1


def band_to_dense(tab, q, K, cols, off):
    """tab[j][r] = M[r][r + off + j - K] -> dense q x cols."""
    D = np.zeros((q, cols))
    P = 2 * K + 1
    for j in range(P):
        for r in range(q):
            c = r + off + j - K
            if 0 <= c < cols:
                D[r, c] = tab[j, r]
            else:
                assert tab[j, r] == 0.0
    return D


CASES = [(k, bc, dom) for k in (0, 1, 2, 3, 4) for bc in ("dirichlet", "neumann") for dom in ("one", "two")]


@pytest.mark.parametrize("k,bc,dom", CASES)
def test_host_tables_match_oracle(mofem, k, bc, dom):
    g1, g2 = (ZERO, SIN_TOP) if dom == "one" else (Profile(c2=0.1), Profile(c0=1.0, ca=0.2, cf=1.0))
    d = max(k, 1)
    n = 6 * d + 1 if k != 3 else 19
    gamma = 0.7
    t = mofem.host_tables(g1, g2, k, n, gamma, bc=0 if bc == "dirichlet" else 1)
    P = Problem(g1, g2, k, n, gamma, bc=bc)
    terms = P.terms()
    keep = [0, 1, 3, 6, 7] if dom == "one" else list(range(8))
    assert t["n_terms"] == len(keep)
    q, K = P.q, t["K"]
    scale = max(abs(S).max() for S, _ in terms)
    for ci, oi in enumerate(keep):
        S, T = terms[oi]
        Sd = band_to_dense(t["S"][ci], q, K, q, 0)
        Td = band_to_dense(t["T"][ci], q, K, q, 0)
        assert np.abs(Sd - S.toarray()).max() <= 1e-12 * max(1.0, abs(S).max())
        assert np.abs(Td - T.toarray()).max() <= 1e-12 * max(1.0, abs(T).max())
    Ms, Mt = P.rhs_factors()
    off = 1 if bc == "dirichlet" else 0
    assert np.abs(band_to_dense(t["Srh"], q, K, n, off) - Ms.toarray()).max() <= 1e-14 * n
    assert np.abs(band_to_dense(t["Trh"], q, K, n, off) - Mt.toarray()).max() <= 1e-14 * n


def test_dib_equilibrium_matches_oracle(mofem):
    """Host Newton of the library vs the oracle's (cap and jar parameters; C = 4 gives (0, 1/2))."""
    from oracle import dib
    for p in (dib.CAP, dib.JAR, dict(dib.CAP, C=4.0)):
        e, t = mofem.dib_equilibrium(p)
        eo, to = dib.equilibrium(p)
        assert abs(e - eo) <= 1e-13 and abs(t - to) <= 1e-13
    # D = 3.2727 is printed to 4 decimals: g(0, 1/2) = 1.5e-5, so the zero moves by O(1e-5 / |J|)
    e, t = mofem.dib_equilibrium(dict(dib.CAP, C=4.0))
    assert abs(e) <= 1e-4 and abs(t - 0.5) <= 1e-4


def test_group_layout_on_host(mofem):
    """Problems of equal (k, n, bc) share a group; groups ordered by decreasing n^3 * size."""
    P = lambda k, n, bc="dirichlet": dict(g1=ZERO, g2=SIN_TOP, k=k, n=n, gamma=1.0, bc=bc)
    probs = [P(2, 33), P(1, 65), P(2, 33), P(2, 33, "neumann"), P(1, 65), P(4, 129), P(2, 33)]
    ng, of = mofem.group_layout(probs)
    assert ng == 4
    assert of[0] == of[2] == of[6] and of[1] == of[4]
    assert len({of[0], of[1], of[3], of[5]}) == 4
    assert of[5] == 0                      # 129^3 x 1 is the most work
    assert mofem.LIB.mofem_group_layout(0, None, None, None) == 1
