"""Closed-form reduced solve for P1 with Dirichlet BC on the unit square (oracle).

Test infrastructure only.

Sec. 4.1: for P1 elements with zero Dirichlet data on [0,1]^2 (N intervals,
q = N - 1 interior nodes) the 1D matrices are tridiagonal Toeplitz,
A = N tridiag(-1, 2, -1) and M = (1/(6N)) tridiag(1, 4, 1), and
M = alpha A + beta I with alpha = -1/(6 N^2), beta = 1/N
(Eq. dirichlet_linear_combination).  A, M and M^{-1}A share the sine
eigenvectors v_i[j] = sin(i j pi / N) (Eq. dirichlet_eigenvectors).

Reading of Eq. dirichlet_eigenvalues: for A = N tridiag(-1, 2, -1) the
eigenvalues are 2N (1 - cos(i pi / N)); the printed factor 2/N belongs to the
unscaled tridiag(-1,2,-1)/N and would be inconsistent with A's definition in
Eq. stiffness_mass_1D.  Eq. dirichlet_combined_eigenvalues is the eigenvalue of
Z1 = M^{-1}A + gamma/2 I:  lambda = lamA / (alpha lamA + beta) + gamma/2,
which with alpha and beta above equals
((12 N^2 - gamma) lamA + 6 N gamma) / (12 N - 2 lamA) as printed.
"""
import numpy as np


def eigen(N, gamma):
    """(X, lam): sine eigenvectors (columns) and the eigenvalues of Z1 = Z2."""
    i = np.arange(1, N)
    lamA = 2.0 * N * (1.0 - np.cos(i * np.pi / N))
    lam = ((12.0 * N * N - gamma) * lamA + 6.0 * N * gamma) / (12.0 * N - 2.0 * lamA)
    X = np.sin(np.outer(i, i) * np.pi / N)
    return X, lam


def solve_square(N, gamma, F_int):
    """U solving (A + g/2 M) U M + M U (A + g/2 M) = M F M, F_int interior nodal f.

    Eq. laplace_dirichlet_sylvester with the Dirichlet-trimmed M F M
    (Eq. neumann_sylvester_0 divides by M on both sides: Z1 U + U Z2 = F), solved
    by Eq. reduced_formula_for_u with X^{-1} = (2/N) X (orthogonality of the
    discrete sine transform).
    """
    X, lam = eigen(N, gamma)
    Xinv = (2.0 / N) * X
    Fh = Xinv @ F_int @ X
    Uh = Fh / (lam[:, None] + lam[None, :])
    return X @ Uh @ Xinv
