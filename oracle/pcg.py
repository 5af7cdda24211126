"""MO-PCG and its preconditioners (oracle; test infrastructure only).

Sec. 5, Eqs. laplace_xnormal_pcg and laplace_xnormal_pcg_iteration define a
matrix-oriented PCG with Frobenius inner products <A, B> = sum(sum(A o B)).  The
printed alpha, beta and search-direction updates are not those of PCG (alpha
uses <Q,R>/<L(Q),R> and the direction update reads Q - beta Q); the paper cites
the standard method (Golub & Van Loan; Saad) and states MO-PCG is equivalent to
vector PCG, so the standard recurrences are used:

    alpha = <R, Z> / <Q, L(Q)>,   U += alpha Q,   R -= alpha L(Q),
    Z = P^{-1}(R),  beta = <R_new, Z_new> / <R, Z>,   Q = Z + beta Q.

Stopping rule: ||R||_F <= rtol ||B||_F (relative residual), with the
recursively updated residual; the elliptic rule of the paper needs the direct
solver's error and is for illustration only.

Preconditioners:
* :class:`ReducedSylvester` -- the two-term Sylvester solve by the reduced
  (spectral) approach of Sec. 4, Eqs. diagonalisation_1 and
  reduced_formula_for_u, on the symmetric-definite pencils, giving
  Z = Q1 ((Q1^T R Q2) ./ (lambda_a + mu_b)) Q2^T.
* :class:`ProductPreconditioner` -- the paper's single-term preconditioner of
  Sec. 5, Eq. vector_preconditioner: Z = E^{-1} R F^{-T}.
* ``AUA`` is the square-domain special case, Eq. precSquare.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla


def fro(A, B):
    """Frobenius inner product sum(sum(A o B))."""
    return float(np.sum(A * B))


class ReducedSylvester:
    """Z solving E1 Z F1^T + E2 Z F2^T = R via generalized eigendecompositions.

    E1 Q1 = E2 Q1 diag(lam), Q1^T E2 Q1 = I;  F2 Q2 = F1 Q2 diag(mu), Q2^T F1 Q2 = I.
    Then E1 = Q1^{-T} Lam Q1^{-1}, E2 = Q1^{-T} Q1^{-1} (likewise for F), so the
    equation becomes Lam Zh + Zh Mu = Q1^T R Q2 with Zh = Q1^{-1} Z Q2^{-T}: the
    Hadamard-divide solve of Sec. 4 (Eq. reduced_formula_for_u).
    """

    def __init__(self, E1, E2, F1, F2):
        self.lam, self.Q1 = sla.eigh(E1, E2)
        self.mu, self.Q2 = sla.eigh(F2, F1)
        self.den = self.lam[:, None] + self.mu[None, :]

    def __call__(self, R):
        W = (self.Q1.T @ R @ self.Q2) / self.den
        return self.Q1 @ W @ self.Q2.T


class ProductPreconditioner:
    """Z = E^{-1} R F^{-T} (Eq. vector_preconditioner; also AUA with E = F = A)."""

    def __init__(self, E, F):
        self.Elu = spla.splu(E.tocsc())
        self.Flu = spla.splu(F.tocsc())

    def __call__(self, R):
        Y = self.Elu.solve(np.asarray(R, dtype=np.float64))           # Y = E^{-1} R
        # Z F^T = Y  <=>  F Z^T = Y^T
        return self.Flu.solve(np.ascontiguousarray(Y.T)).T


def mo_pcg(apply, precond, B, U0=None, rtol=1e-10, max_iter=1000, record=False):
    """Matrix-oriented PCG (standard recurrences, see module docstring).

    Returns (U, info) with info = {'iterations', 'rel_residual', 'history'}.
    ``history`` (if ``record``) holds U after every iteration.
    """
    B = np.asarray(B, dtype=np.float64)
    U = np.zeros_like(B) if U0 is None else np.array(U0, dtype=np.float64)
    R = B - apply(U)
    nb = np.sqrt(fro(B, B))
    hist = []
    if nb == 0.0:
        return U, {'iterations': 0, 'rel_residual': 0.0, 'history': hist}
    Z = precond(R)
    Q = Z.copy()
    rz = fro(R, Z)
    it = 0
    rel = np.sqrt(fro(R, R)) / nb
    while rel > rtol and it < max_iter:
        LQ = apply(Q)
        alpha = rz / fro(Q, LQ)
        U = U + alpha * Q
        R = R - alpha * LQ
        it += 1
        if record:
            hist.append(U.copy())
        rel = np.sqrt(fro(R, R)) / nb
        if rel <= rtol:
            break
        Z = precond(R)
        rz_new = fro(R, Z)
        beta = rz_new / rz
        rz = rz_new
        Q = Z + beta * Q
    return U, {'iterations': it, 'rel_residual': rel, 'history': hist}


def vector_pcg(K, Pinv, b, rtol=1e-10, max_iter=1000, record=False):
    """Classical vector PCG on K x = b with preconditioner solve Pinv(r).

    The comparison system of Sec. 5 ("Matrix PCG vs. classical PCG"); here it
    only pins the equivalence of MO-PCG iterates with vec-form PCG.
    """
    x = np.zeros_like(b)
    r = b - K @ x
    nb = np.linalg.norm(b)
    z = Pinv(r)
    p = z.copy()
    rz = r @ z
    hist = []
    it = 0
    while np.linalg.norm(r) / nb > rtol and it < max_iter:
        Kp = K @ p
        alpha = rz / (p @ Kp)
        x = x + alpha * p
        r = r - alpha * Kp
        it += 1
        if record:
            hist.append(x.copy())
        if np.linalg.norm(r) / nb <= rtol:
            break
        z = Pinv(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, {'iterations': it, 'history': hist}


def solve(problem, F, precond='reduced', rtol=1e-13, max_iter=5000, U0=None, pencil='averaged'):
    """Reference solve of the MO-FEM system for nodal f = F (n x n).

    ``precond``: 'reduced' (two-term Sylvester, reduced approach) or 'product'
    (the paper's single-term preconditioner).
    """
    from .operator import apply_terms, rhs
    terms = [(S, T) for S, T in problem.terms() if S.nnz and abs(S).sum() > 0]
    B = rhs(problem, F)
    if precond == 'reduced':
        P = ReducedSylvester(*problem.pencils(pencil))
    elif precond == 'product':
        P = ProductPreconditioner(*problem.product_factors())
    else:
        raise ValueError(precond)
    return mo_pcg(lambda X: apply_terms(terms, X), P, B, U0=U0, rtol=rtol, max_iter=max_iter)
