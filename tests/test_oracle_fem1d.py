"""Pins for oracle.fem1d: 1D bases, quadrature and weighted 1D matrices.

Pins (none re-types the code under test):
* Lagrange basis: Kronecker-delta at the nodes, partition of unity, derivative
  checked against a central finite difference.
* Gauss rule: exact on monomials up to degree 2 nq - 1 (closed form 1/(p+1)).
* P1 closed forms of Sec. 4.1 (Eq. dirichlet_linear_combination):
  A = N tridiag(-1, 2, -1), M = tridiag(1, 4, 1)/(6N), M = alpha A + beta I with
  alpha = -1/(6 N^2), beta = 1/N after Dirichlet trimming.
* Lumped P1 (Sec. 3.3): M0 diagonal with m0 = 1/N on interior nodes
  (Eq. dirichlet_lumped_constant); the Dirichlet-trimmed convection matrix is
  Toeplitz and skew-symmetric (Eq. dirichlet_convection_skew_symmetric).
* Invariants for any weight: sum_ij M[w]_ij = int w (partition of unity),
  K[w] 1 = 0, 1^T G[w] = 0 and G[w] 1 = (int psi_i' w)_i; K[w] and M[w]
  symmetric; for polynomial w exact against sympy-free closed forms.
"""
import numpy as np
import pytest

from oracle.fem1d import lagrange_ref, quadrature, Mesh1D, interior, trim


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_lagrange_nodal_and_partition(k):
    nodes = np.arange(k + 1) / k
    phi, dphi = lagrange_ref(k, nodes)
    assert np.allclose(phi, np.eye(k + 1), atol=1e-13)
    x = np.linspace(0, 1, 37)
    phi, dphi = lagrange_ref(k, x)
    assert np.allclose(phi.sum(0), 1.0, atol=1e-13)
    assert np.allclose(dphi.sum(0), 0.0, atol=1e-11)
    eps = 1e-6
    pp, _ = lagrange_ref(k, x + eps)
    pm, _ = lagrange_ref(k, x - eps)
    assert np.allclose((pp - pm) / (2 * eps), dphi, atol=1e-6)


@pytest.mark.parametrize("nq", [2, 3, 5, 7])
def test_gauss_exactness(nq):
    x, w = quadrature(1, nq)
    for p in range(2 * nq):
        assert abs(np.sum(w * x ** p) - 1.0 / (p + 1)) < 1e-14


def test_p1_closed_forms():
    N = 10
    m = Mesh1D(N + 1, 1)
    i = interior(N + 1, 'dirichlet')
    A = trim(m.matrix('K', None), i).toarray()
    M = trim(m.matrix('M', None), i).toarray()
    q = N - 1
    T = lambda a, b, c: a * np.eye(q, k=-1) + b * np.eye(q) + c * np.eye(q, k=1)
    assert np.allclose(A, N * T(-1, 2, -1), atol=1e-12)
    assert np.allclose(M, T(1, 4, 1) / (6 * N), atol=1e-14)
    alpha, beta = -1.0 / (6 * N * N), 1.0 / N
    assert np.allclose(M, alpha * A + beta * np.eye(q), atol=1e-14)


def test_lumped_p1():
    N = 12
    m = Mesh1D(N + 1, 0)
    i = interior(N + 1, 'dirichlet')
    M0 = trim(m.matrix('M', None), i).toarray()
    assert np.allclose(M0, np.eye(N - 1) / N, atol=1e-15)
    # lumped stiffness = exact P1 stiffness (psi' psi' is constant per element)
    A0 = trim(m.matrix('K', None), i).toarray()
    A1 = trim(Mesh1D(N + 1, 1).matrix('K', None), i).toarray()
    assert np.allclose(A0, A1, atol=1e-12)
    C = trim(m.matrix('G', None), i).toarray()
    assert np.allclose(C.T, -C, atol=1e-15)
    assert np.allclose(np.diag(C, 1), np.diag(C, 1)[0]) and abs(np.diag(C, 1)[0] + 0.5) < 1e-15
    # lumped weighted mass = diag(w(x_i)) * m0 (nodal quadrature of Sec. 3.3)
    w = lambda x: 1.0 + 0.5 * np.sin(3 * x)
    Mw = trim(m.matrix('M', w), i).toarray()
    assert np.allclose(Mw, np.diag(w(m.nodes[i])) / N, atol=1e-15)


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_weighted_invariants(k):
    deg = max(k, 1)
    n = 6 * deg + 1
    m = Mesh1D(n, k)
    w = lambda x: 1.0 + x + 0.3 * np.cos(2 * x)
    K, M, G = (m.matrix(c, w).toarray() for c in 'KMG')
    one = np.ones(n)
    assert np.allclose(K, K.T, atol=1e-13) and np.allclose(M, M.T, atol=1e-15)
    assert np.allclose(K @ one, 0.0, atol=1e-11)
    assert np.allclose(one @ G, 0.0, atol=1e-12)
    # polynomial weight: total mass = int_0^1 (1 + x + x^2) = 11/6 (exact for P_k, nq = k+3)
    if k > 0:
        Mp = m.matrix('M', lambda x: 1 + x + x * x).toarray()
        assert abs(Mp.sum() - 11.0 / 6.0) < 1e-13
        # G[1] 1 = int psi_i' : -1 at node 0, +1 at node n-1, 0 elsewhere
        g = m.matrix('G', None).toarray() @ one
        e = np.zeros(n); e[0], e[-1] = -1.0, 1.0
        assert np.allclose(g, e, atol=1e-12)
        # quadratic form of K[x^2] on the interpolant of x^2: int (2x)^2 x^2 = 4/5 (k >= 2 exact)
        if k >= 2:
            v = m.nodes ** 2
            assert abs(v @ m.matrix('K', lambda x: x * x).toarray() @ v - 0.8) < 1e-12
