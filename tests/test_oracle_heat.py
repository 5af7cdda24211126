"""Pins of the oracle's IMEX Euler heat solver and its discrete adjoint (CPU).

* Forward: on the unit square with P1 and Dirichlet BC a separable sine mode
  v_i v_j^T is an eigenvector of M~^{-1} A~ with eigenvalue lam_i + lam_j (the 1D
  eigenvalues of M^{-1} A, Sec. 4.1 with the corrected Eq. dirichlet_eigenvalues),
  so N steps multiply it by (1 + d tau (lam_i + lam_j))^{-N} exactly.
* d_u gradient: for that mode and J = ||U_N - c0 U_0||^2 the derivative is a
  closed form in d.
* Adjoint against the forward map: on curved two-profile domains (eight terms,
  Dirichlet and Neumann, P1/P2) the adjoint gradient equals central finite
  differences of the forward solve, for U_0 along random directions and for d_u.
"""
import numpy as np
import pytest

from oracle import closed_form
from oracle.heat import HeatOperators, imex_forward, imex_adjoint, loss
from paper_2109_01173_gb300.inputs import Profile, ZERO

ONE = Profile(c0=1.0)
G1 = Profile(c2=0.1)                      # 0.1 x^2
G2 = Profile(c0=1.0, ca=0.2, cf=1.0)      # 1 + 0.2 cos(pi x)


def _mode(N, i, j):
    X, lam = closed_form.eigen(N, 0.0)    # columns: sine vectors, lam: eigenvalues of M^-1 A
    return np.outer(X[:, i - 1], X[:, j - 1]), lam[i - 1] + lam[j - 1]


def test_square_mode_decays_by_the_closed_form_factor():
    N, d, tau, steps = 16, 0.3, 0.01, 7
    ops = HeatOperators(ZERO, ONE, 1, N + 1, 'dirichlet')
    U0, Lam = _mode(N, 2, 3)
    UN = imex_forward(ops, d, tau, U0, steps)[-1]
    factor = (1.0 + d * tau * Lam) ** (-steps)
    assert np.abs(UN - factor * U0).max() <= 1e-12 * np.abs(U0).max()


def test_square_du_gradient_closed_form():
    N, d, tau, steps, c0 = 12, 0.2, 0.02, 5, 0.5
    ops = HeatOperators(ZERO, ONE, 1, N + 1, 'dirichlet')
    U0, Lam = _mode(N, 1, 2)
    states = imex_forward(ops, d, tau, U0, steps)
    J, dJ = loss(states[-1], c0 * U0)
    _, g_du = imex_adjoint(ops, d, tau, states, dJ)
    c = (1.0 + d * tau * Lam) ** (-steps)
    dc = -steps * tau * Lam * (1.0 + d * tau * Lam) ** (-steps - 1)
    expect = 2.0 * (c - c0) * dc * float(np.sum(U0 * U0))
    assert abs(J - (c - c0) ** 2 * float(np.sum(U0 * U0))) <= 1e-12 * J
    assert abs(g_du - expect) <= 1e-10 * abs(expect)


@pytest.mark.parametrize("k,n,bc", [(1, 9, "dirichlet"), (2, 9, "neumann"), (2, 7, "dirichlet"), (0, 8, "neumann")])
def test_adjoint_equals_central_differences(k, n, bc):
    d, tau, steps = 0.05, 2e-2, 6
    ops = HeatOperators(G1, G2, k, n, bc)
    q = ops.q
    rng = np.random.default_rng(10 * k + n)
    U0 = rng.uniform(0, 1, (q, q))
    T = rng.uniform(0, 1, (q, q))

    def J_of(U, dd):
        return loss(imex_forward(ops, dd, tau, U, steps)[-1], T)[0]

    states = imex_forward(ops, d, tau, U0, steps)
    _, dJ = loss(states[-1], T)
    gU, g_du = imex_adjoint(ops, d, tau, states, dJ)
    # U_0 directions: J is quadratic in U_0, central differences are exact up to rounding
    for _ in range(3):
        V = rng.standard_normal((q, q))
        eps = 1e-3
        fd = (J_of(U0 + eps * V, d) - J_of(U0 - eps * V, d)) / (2 * eps)
        assert abs(fd - float(np.sum(gU * V))) <= 1e-8 * max(abs(fd), 1e-12) + 1e-12
    eps = 1e-5 * d
    fd = (J_of(U0, d + eps) - J_of(U0, d - eps)) / (2 * eps)
    assert abs(fd - g_du) <= 1e-6 * abs(fd)
