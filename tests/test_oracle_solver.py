"""Pins for oracle.pcg and oracle.closed_form (the solver's result and iterates).

* MO-PCG (reduced and product preconditioners) reaches the direct solution of
  the independent vector-form system (Sec. 5: MO and vector forms give the same
  solution up to rounding).
* MO-PCG iterates equal vector-PCG iterates on vec(U) with the Kronecker
  preconditioner (Sec. 5, "Matrix PCG vs. classical PCG": the methods are
  equivalent).
* The reduced-approach preconditioner solves its two-term Sylvester equation
  (Sec. 4, Eq. reduced_formula_for_u); on the square it is the whole operator,
  so MO-PCG stops after one iteration.
* Closed-form P1 Dirichlet reduced solve on the square (Sec. 4.1) equals the
  direct solve.
* Convergence orders on manufactured solutions: k + 1 (k = 2: 4, superconvergent,
  Sec. 4.2) and quadratic P1 on the cap domain (Sec. 5.2).
* The paper's printed iteration count: AUA on the square stops after two
  iterations under the increment rule (Sec. 5.1, Table 1).
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.operator import Problem, apply_terms, rhs
from oracle.fem1d import trim
from oracle import pcg, assembly2d, closed_form
from paper_2109_01173_gb300.inputs import Profile, ZERO, SIN_TOP, manufactured_sin_f, fourier_f

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_printed_values.json")))
TWO = (Profile(c2=0.1), Profile(c0=1.0, ca=0.2, cf=1.0))


def live_terms(P):
    return [(S, T) for S, T in P.terms() if abs(S).sum() > 0]


# the single-term product preconditioner K_s (x) K_t is singular under Neumann (constants
# are in the kernel of both stiffness factors): that pairing is not a case
_BC_PRECOND = [(bc, gamma, pre) for bc, gamma in (("dirichlet", 0.0), ("dirichlet", 2.0), ("neumann", 1.0))
               for pre in ("reduced", "product") if not (pre == "product" and bc == "neumann")]


@pytest.mark.parametrize("k,n", [(0, 11), (1, 11), (2, 11), (4, 13)])
@pytest.mark.parametrize("bc,gamma,precond", _BC_PRECOND)
def test_pcg_matches_direct(k, n, bc, gamma, precond):
    P = Problem(*TWO, k, n, gamma=gamma, bc=bc)
    F = np.random.default_rng(3).standard_normal((n, n))
    Ud = assembly2d.direct_solve(P, F)
    U, info = pcg.solve(P, F, precond=precond, rtol=1e-13, max_iter=2000)
    assert np.linalg.norm(U - Ud) <= 1e-10 * np.linalg.norm(Ud)
    assert info['rel_residual'] <= 1e-13


def test_product_factors_singular_under_neumann():
    """Why the product preconditioner has no Neumann case: both of its factors annihilate
    the constant vector (stiffness row sums vanish without Dirichlet trimming)."""
    P = Problem(*TWO, 2, 11, gamma=1.0, bc="neumann")
    E, F = P.product_factors()
    one = np.ones(P.q)
    assert np.abs(E @ one).max() <= 1e-12 * abs(E).max()
    assert np.abs(F @ one).max() <= 1e-12 * abs(F).max()


def test_mo_pcg_iterates_equal_vector_pcg():
    P = Problem(*TWO, 2, 9, gamma=1.0)
    F = np.random.default_rng(4).standard_normal((P.n, P.n))
    E1, E2, F1, F2 = P.pencils()
    Pmat = np.kron(E1, F1) + np.kron(E2, F2)
    K, Mr = assembly2d.system(P)
    b = Mr @ F.ravel()
    x, vinfo = pcg.vector_pcg(K, lambda r: np.linalg.solve(Pmat, r), b, rtol=1e-12, record=True)
    Pc = pcg.ReducedSylvester(E1, E2, F1, F2)
    U, minfo = pcg.mo_pcg(lambda X: apply_terms(live_terms(P), X), Pc, rhs(P, F), rtol=1e-12, record=True)
    assert minfo['iterations'] == vinfo['iterations']
    for Ui, xi in zip(minfo['history'], vinfo['history']):
        assert np.linalg.norm(Ui.ravel() - xi) <= 1e-9 * np.linalg.norm(xi)


@pytest.mark.parametrize("variant", ["dominant", "averaged"])
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_reduced_preconditioner_solves_sylvester(variant, bc):
    P = Problem(*TWO, 3, 19, gamma=0.5, bc=bc)
    E1, E2, F1, F2 = P.pencils(variant)
    Pc = pcg.ReducedSylvester(E1, E2, F1, F2)
    R = np.random.default_rng(6).standard_normal((P.q, P.q))
    Z = Pc(R)
    back = E1 @ Z @ F1.T + E2 @ Z @ F2.T
    assert np.linalg.norm(back - R) <= 1e-11 * np.linalg.norm(R)
    # Q1^T E2 Q1 = I and Q2^T F1 Q2 = I (normalisation used by the Hadamard solve)
    assert np.allclose(Pc.Q1.T @ E2 @ Pc.Q1, np.eye(P.q), atol=1e-9)
    assert np.allclose(Pc.Q2.T @ F1 @ Pc.Q2, np.eye(P.q), atol=1e-9)


@pytest.mark.parametrize("k", [1, 2, 4])
def test_square_one_iteration(k):
    P = Problem(ZERO, Profile(c0=1.0), k, 8 * k + 1, gamma=0.7)
    F = np.random.default_rng(7).standard_normal((P.n, P.n))
    U, info = pcg.solve(P, F, rtol=1e-12)
    assert info['iterations'] == 1


def test_closed_form_p1_square():
    N, gamma = 16, 3.0
    P = Problem(ZERO, Profile(c0=1.0), 1, N + 1, gamma=gamma)
    s = np.arange(N + 1) / N
    F = np.outer(np.sin(2 * np.pi * s), np.sin(np.pi * s) * (1 + s))   # zero on the boundary
    Ucf = closed_form.solve_square(N, gamma, F[1:-1, 1:-1])
    Ud = assembly2d.direct_solve(P, F)
    assert np.linalg.norm(Ucf - Ud) <= 1e-12 * np.linalg.norm(Ud)


def rate(errs):
    return np.log2(np.array(errs[:-1]) / np.array(errs[1:]))


def nodal_l2(P, E):
    f = P.factors()
    Ms, Mt = trim(f['Ms_h'], P.idx), trim(f['Mt'], P.idx)
    return np.sqrt(np.sum(E * (Ms @ E @ Mt.T)))


@pytest.mark.parametrize("k,order", [(0, 2), (1, 2), (2, 4), (3, 4)])
def test_manufactured_rates_sin_domain(k, order):
    errs = []
    for E in (8, 16, 32):
        n = E * max(k, 1) + 1
        P = Problem(ZERO, SIN_TOP, k, n, gamma=1.0)
        F, u = manufactured_sin_f(ZERO, SIN_TOP, n, 1.0)
        U, _ = pcg.solve(P, F, rtol=1e-13)
        errs.append(nodal_l2(P, U - u[1:-1, 1:-1]))
    r = rate(errs)
    assert r[-1] > order - 0.25, r


def _pmul(a, b):
    out = np.zeros((a.shape[0] + b.shape[0] - 1, a.shape[1] + b.shape[1] - 1))
    for i in range(a.shape[0]):
        for j in range(a.shape[1]):
            out[i:i + b.shape[0], j:j + b.shape[1]] += a[i, j] * b
    return out


def test_cap_domain_p1_quadratic():
    """Sec. 5.2 exact solution, written in this orientation (x <-> y swapped)."""
    P2 = np.polynomial.polynomial
    # u = x (x - 1) (-x^2/2 + y + 1) (x^2/2 + y - 1); coefficient arrays c[i, j] of x^i y^j
    f1 = np.array([[0.0], [-1.0], [1.0]])
    f2 = np.array([[1.0, 1.0], [0.0, 0.0], [-0.5, 0.0]])
    f3 = np.array([[-1.0, 1.0], [0.0, 0.0], [0.5, 0.0]])
    c = _pmul(_pmul(f1, f2), f3)
    lap = P2.polyder(c, 2, axis=0)
    lap = np.pad(lap, ((0, 2), (0, 0))) + np.pad(P2.polyder(c, 2, axis=1), ((0, 0), (0, 2)))
    g1, g2 = Profile(c0=-1.0, c2=0.5), Profile(c0=1.0, c2=-0.5)
    errs = []
    for N in (12, 24, 48):
        n = N + 1
        s = np.arange(n) / N
        X = np.repeat(s[:, None], n, 1)
        Y = g1.g(s)[:, None] + s[None, :] * (g2.g(s) - g1.g(s))[:, None]
        F = -P2.polyval2d(X, Y, lap)
        u = P2.polyval2d(X, Y, c)
        P = Problem(g1, g2, 1, n, gamma=0.0)
        U, _ = pcg.solve(P, F, rtol=1e-13)
        errs.append(nodal_l2(P, U - u[1:-1, 1:-1]))
    r = rate(errs)
    assert abs(r[-1] - GOLD['cap_domain_p1_order']['value']) < 0.1, r


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_paper_aua_two_iterations(k):
    N = 24
    n = N + 1
    P = Problem(ZERO, Profile(c0=1.0), k, n, gamma=0.0)
    s = np.arange(n) / N
    F = 8 * np.pi ** 2 * np.outer(np.sin(2 * np.pi * s), np.sin(2 * np.pi * s))
    Uex = np.outer(np.sin(2 * np.pi * s), np.sin(2 * np.pi * s))[1:-1, 1:-1]
    errv = np.linalg.norm(assembly2d.direct_solve(P, F) - Uex)
    A = trim(P.factors()['Kt_1'], P.idx)
    U, info = pcg.mo_pcg(lambda X: apply_terms(live_terms(P), X), pcg.ProductPreconditioner(A, A),
                         rhs(P, F), rtol=1e-15, max_iter=10, record=True)
    hist = [np.zeros_like(U)] + info['history']
    stop = next(i for i in range(1, len(hist)) if np.linalg.norm(hist[i] - hist[i - 1]) <= 0.05 * errv)
    assert stop == GOLD['square_aua_pcg_iterations']['value']


@pytest.mark.parametrize("k,n", [(0, 11), (1, 11), (2, 11), (4, 13)])
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_averaged_pencil_is_the_t_mean_of_the_operator_terms(k, n, bc):
    """The 'averaged' second pencil E2 = M_s[e2] is the mean over t in [0, 1] of the
    operator's K_t-paired s-factors.  H^_tt = (1 + (g1' + t h')^2)/h splits as
    (1 + g1'^2)/h + t (2 g1' h'/h) + t^2 (h'^2/h), which the operator pairs with K_t[1],
    K_t[t] and K_t[t^2] (terms 1, 2, 3); replacing t and t^2 by their means 1/2 and 1/3
    gives M_s[e2] = S_1 + S_2 / 2 + S_3 / 3 exactly, with the S_i of terms() (pinned
    against the physical-mesh 2D assembly).  Two curved profiles, so every piece is
    nonzero."""
    P = Problem(*TWO, k, n, gamma=1.0, bc=bc)
    t = P.terms()
    assert min(abs(t[i][0]).sum() for i in (1, 2, 3)) > 0
    E2 = P.pencils('averaged')[1]
    want = (t[1][0] + 0.5 * t[2][0] + t[3][0] / 3.0).toarray()
    assert np.abs(E2 - want).max() <= 1e-13 * np.abs(want).max()
    # and it is not the 'dominant' (t-free) pencil on this domain
    assert np.abs(P.pencils('dominant')[1] - want).max() > 1e-6 * np.abs(want).max()
