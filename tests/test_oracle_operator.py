"""Pins for oracle.operator (Kronecker operator) and oracle.assembly2d.

* The eight-term Kronecker operator equals the independent physical-mesh 2D
  vector-form assembly (Eq. laplace_xnormal_FEM) to 1e-12 for k = 0..4, both
  boundary conditions, with one (5-term) and two (8-term) curved profiles.
* The 2D assembly itself is pinned by closed forms: total mass = area of the
  domain, the energy of a linear function equals |grad u|^2 * area (patch test),
  and on the unit square it equals A (x) M + M (x) A with the P1 closed forms
  (Eq. kronecker_mass).
* Invariants of the operator: symmetry and positive definiteness (Sec. 5:
  A~ + gamma M~ is SPD); on the square the cross and t-weighted terms vanish
  (Sec. 3.2 remark after Eq. kronecker_mass_distorted).
"""
import numpy as np
import pytest

from oracle.operator import Problem, apply_terms, rhs, apply_entry
from oracle import assembly2d
from paper_2109_01173_gb300.inputs import Profile, ZERO, SIN_TOP

TWO = (Profile(c2=0.1), Profile(c0=1.0, ca=0.2, cf=1.0))      # 0.1x^2 <= y <= 1 + 0.2 cos(pi x)
ONE = (ZERO, SIN_TOP)                                           # 0 <= y <= 1 + 0.25 sin(2 pi x)


def kron_matrix(P):
    terms = P.terms()
    q = P.q
    L = np.zeros((q * q, q * q))
    for j in range(q * q):
        e = np.zeros(q * q)
        e[j] = 1.0
        L[:, j] = apply_terms(terms, e.reshape(q, q)).ravel()
    return L


@pytest.mark.parametrize("dom", [ONE, TWO], ids=["one_profile", "two_profiles"])
@pytest.mark.parametrize("k,n", [(0, 9), (1, 9), (2, 9), (3, 10), (4, 9)])
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_kronecker_equals_2d_assembly(dom, k, n, bc):
    P = Problem(dom[0], dom[1], k, n, gamma=0.7, bc=bc)
    K, Mr = assembly2d.system(P)
    L = kron_matrix(P)
    assert np.abs(L - K.toarray()).max() <= 1e-12 * np.abs(L).max()
    F = np.random.default_rng(1).standard_normal((n, n))
    b1 = rhs(P, F).ravel()
    b2 = Mr @ F.ravel()
    assert np.abs(b1 - b2).max() <= 1e-12 * np.abs(b1).max()


def test_five_terms_when_lower_profile_is_flat():
    P = Problem(*ONE, 2, 9, gamma=1.0)
    zero = [i for i, (S, T) in enumerate(P.terms()) if abs(S).sum() == 0]
    assert zero == [2, 4, 5]


def test_square_reduces_to_sylvester():
    N = 8
    P = Problem(ZERO, Profile(c0=1.0), 1, N + 1, gamma=0.5)
    t = P.terms()
    for i in range(2, 8):
        assert abs(t[i][0]).sum() < 1e-14
    q = N - 1
    T = lambda a, b, c: a * np.eye(q, k=-1) + b * np.eye(q) + c * np.eye(q, k=1)
    A, M = N * T(-1, 2, -1), T(1, 4, 1) / (6 * N)
    assert np.allclose(t[0][0].toarray(), A + 0.5 * M, atol=1e-12)
    assert np.allclose(t[0][1].toarray(), M, atol=1e-14)
    assert np.allclose(t[1][0].toarray(), M, atol=1e-14)
    assert np.allclose(t[1][1].toarray(), A, atol=1e-12)
    K, _ = assembly2d.system(P)
    assert np.allclose(K.toarray(), np.kron(A, M) + np.kron(M, A) + 0.5 * np.kron(M, M), atol=1e-12)


def test_2d_mass_is_area_and_patch_test():
    # quadratic profiles: y = g1(s) + t h(s) lies in the Q2 space, h is polynomial
    g1, g2 = Profile(c2=0.1), Profile(c0=1.0, c2=0.2)
    area = 1.0 + (0.2 - 0.1) / 3.0
    P = Problem(g1, g2, 2, 9, gamma=0.0, bc='neumann')
    K, M = assembly2d.assemble(P)
    one = np.ones(P.n * P.n)
    assert abs(one @ M @ one - area) < 1e-13
    X = np.repeat((np.arange(P.n) / (P.n - 1))[:, None], P.n, axis=1)
    s = X[:, 0]
    Y = g1.g(s)[:, None] + (np.arange(P.n) / (P.n - 1))[None, :] * (g2.g(s) - g1.g(s))[:, None]
    for a, b in [(1.0, 0.0), (0.0, 1.0), (0.3, -2.0)]:
        u = (a * X + b * Y + 0.7).ravel()
        assert abs(u @ K @ u - (a * a + b * b) * area) < 1e-11
        assert np.allclose(K @ np.ones_like(u), 0.0, atol=1e-11)


@pytest.mark.parametrize("k", [0, 1, 2, 4])
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_operator_symmetric_positive(k, bc):
    deg = max(k, 1)
    P = Problem(*TWO, k, 4 * deg + 1, gamma=0.3, bc=bc)
    terms = P.terms()
    rng = np.random.default_rng(5)
    X, Y = rng.standard_normal((2, P.q, P.q))
    lhs = np.sum(X * apply_terms(terms, Y))
    rhs_ = np.sum(apply_terms(terms, X) * Y)
    assert abs(lhs - rhs_) <= 1e-12 * abs(lhs)
    assert np.sum(X * apply_terms(terms, X)) > 0


def test_apply_entry_matches_apply():
    P = Problem(*TWO, 3, 13, gamma=1.0)
    terms = P.terms()
    X = np.random.default_rng(2).standard_normal((P.q, P.q))
    Y = apply_terms(terms, X)
    for a, b in [(0, 0), (3, 7), (P.q - 1, P.q - 1), (5, P.q - 1)]:
        assert abs(apply_entry(terms, X, a, b) - Y[a, b]) <= 1e-12 * np.abs(Y).max()
