"""IMEX Euler for the heat equation and its discrete adjoint (oracle).

Test infrastructure only: only tests/, the package's smoke check and the bench's
CPU baseline may import it.

Sec. 6 (Eqs. semilinear_heat_equation_fully_discrete_sylvester_pk and _R_pk):
u_t - d_u Lap u = f(u) with the diffusion implicit and f explicit,

    (M~ + d_u tau A~) U_{n+1} = M~ (U_n + tau F(U_n)),

where, in the matrix-oriented form of Sec. 5, A~ is the multiterm operator
U -> sum_i S_i U T_i^T of the Laplacian (Problem with gamma = 0) and
M~ : U -> M_s[h] U M_t^T the mass operator, both on the interior (Dirichlet) or
all (Neumann) nodes.  Here both are assembled as sparse Kronecker matrices acting
on vec(U) (row-major: kron(S, T) vec(U) = vec(S U T^T)) and every step is a direct
sparse solve: no iteration, no preconditioner.

For f = 0 one step is the linear map U_{n+1} = S^{-1} M U_n with the symmetric
positive definite S = M + d_u tau A.  For a loss J(U_N) of the final state the
discrete adjoint (derived here; the paper does not differentiate) is

    lam_N = dJ/dU_N,
    for n = N-1 .. 0:   y = S^{-1} lam_{n+1},   lam_n = M y,
                        dJ/dd_u += -tau <y, A U_{n+1}>_F,
    dJ/dU_0 = lam_0,

from differentiating S U_{n+1} = M U_n:  S dU_{n+1} = M dU_n - tau dd_u A U_{n+1}.
With a source and a linear reaction, u_t - d_u Lap u = f(x) - r u, both explicit as
Sec. 6 treats the reaction term (f nodal on all n x n nodes, constant in time):

    S U_{n+1} = (1 - tau r) M U_n + tau M_all f,      M_all f := M_s[h]_{int,all} F M_t_{int,all}^T,

and differentiating, S dU_{n+1} = (1 - tau r) M dU_n - tau dr M U_n + tau M_all df
- tau dd_u A U_{n+1}, so with y = S^{-1} lam_{n+1}:

    lam_n = (1 - tau r) M y,   dJ/df += tau M_all^T y,   dJ/dr += -tau <y, M U_n>,
    dJ/dd_u += -tau <y, A U_{n+1}>.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fem1d import trim
from .operator import Problem, apply_terms, rhs
from .pcg import ProductPreconditioner, mo_pcg, fro


def kron_operator(terms):
    """Sparse matrix of U -> sum_i S_i U T_i^T on row-major vec(U)."""
    out = None
    for S, T in terms:
        K = sp.kron(sp.csr_matrix(S), sp.csr_matrix(T), format='csr')
        out = K if out is None else out + K
    return out.tocsc()


class HeatOperators:
    """A (stiffness, gamma = 0) and M (mass) of a domain as sparse q^2 x q^2 matrices."""

    def __init__(self, g1, g2, k, n, bc='dirichlet'):
        P = Problem(g1, g2, k, n, 0.0, bc=bc)
        self.problem = P
        self.q = P.q
        self.A = kron_operator(P.terms())
        f = P.factors()
        self.M = sp.kron(trim(f['Ms_h'], P.idx), trim(f['Mt'], P.idx), format='csc')
        self.M_all = sp.kron(trim(f['Ms_h'], P.idx, np.arange(n)), trim(f['Mt'], P.idx, np.arange(n)),
                             format='csc')

    def system(self, d_u, tau):
        """Factorised S = M + d_u tau A."""
        return spla.splu((self.M + (d_u * tau) * self.A).tocsc())


def imex_forward(ops, d_u, tau, U0, n_steps, F=None):
    """States U_0 .. U_N of IMEX Euler; F(U) -> nodal f on the q x q unknowns (None: f = 0)."""
    lu = ops.system(d_u, tau)
    q = ops.q
    U = np.asarray(U0, dtype=np.float64).reshape(q, q)
    states = [U]
    for _ in range(n_steps):
        rhs_v = U.ravel()
        if F is not None:
            rhs_v = rhs_v + tau * np.asarray(F(U), dtype=np.float64).ravel()
        U = lu.solve(ops.M @ rhs_v).reshape(q, q)
        states.append(U)
    return states


def imex_adjoint(ops, d_u, tau, states, dJ_dUN):
    """(dJ/dU_0, dJ/dd_u) for f = 0 by the discrete adjoint recursion of the module docstring."""
    lu = ops.system(d_u, tau)
    q = ops.q
    lam = np.asarray(dJ_dUN, dtype=np.float64).ravel()
    g_du = 0.0
    for n in range(len(states) - 2, -1, -1):
        y = lu.solve(lam)           # S symmetric: S^T = S
        g_du -= tau * float(y @ (ops.A @ states[n + 1].ravel()))
        lam = ops.M @ y
    return lam.reshape(q, q), g_du


def loss(UN, target):
    """J = ||U_N - U_target||_F^2 and dJ/dU_N."""
    D = np.asarray(UN) - np.asarray(target)
    return float(np.sum(D * D)), 2.0 * D


def paper_heat_preconditioner(problem, d_u, tau):
    """The paper's single-term preconditioner of an IMEX step (Sec. 6, Eq.
    semilinear_heat_equation_fully_discrete_P), P^{-1}(U) = (M3 + d_u tau B1)^{-1} U
    (M + d_u tau (A + B2))^{-1}, in this orientation (the factors of the elliptic
    product preconditioner, Eq. vector_preconditioner, plus the masses):
    (M_s[h] + d_u tau K_s[h])^{-1} U (M_t + d_u tau (K_t + K_t[t^2]))^{-T}."""
    f = problem.factors()
    i = problem.idx
    E = trim(f['Ms_h'], i) + d_u * tau * trim(f['Ks_h'], i)
    F = trim(f['Mt'], i) + d_u * tau * (trim(f['Kt_1'], i) + trim(f['Kt_t2'], i))
    return ProductPreconditioner(E.tocsr(), F.tocsr())


def imex_mo_pcg_step(problem, d_u, tau, U, F_all, precond, max_iter=100):
    """One IMEX Euler step (Sec. 6, Eqs. semilinear_heat_equation_fully_discrete_sylvester_pk
    and _R_pk) by MO-PCG from the guess U_n, stopped by the paper's rule
    ||R_s|| <= tau ||R_0|| (Sec. 6).  F_all: nodal f on all n x n nodes (the load is the
    mass of the interior test functions against it).  `problem` has gamma = 0.
    Returns (U_{n+1}, iterations)."""
    f = problem.factors()
    i = problem.idx
    Ms, Mt = trim(f['Ms_h'], i), trim(f['Mt'], i)
    terms = [(S, T) for S, T in problem.terms() if abs(S).sum() > 0]

    def L(X):
        return Ms @ X @ Mt.T + d_u * tau * apply_terms(terms, X)

    B = Ms @ U @ Mt.T + tau * rhs(problem, F_all)
    R0 = B - L(U)
    nb = np.sqrt(fro(B, B))
    if nb == 0.0:
        return U, 0
    U1, info = mo_pcg(L, precond, B, U0=U, rtol=tau * np.sqrt(fro(R0, R0)) / nb, max_iter=max_iter)
    return U1, info['iterations']


def imex_forward_src(ops, d_u, tau, U0, n_steps, F, r):
    """States U_0 .. U_N of S U_{n+1} = (1 - tau r) M U_n + tau M_all F (module docstring):
    a nodal source F (n x n, constant in time) and a linear reaction r u, both explicit."""
    lu = ops.system(d_u, tau)
    q = ops.q
    U = np.asarray(U0, dtype=np.float64).reshape(q, q)
    src = tau * (ops.M_all @ np.asarray(F, dtype=np.float64).ravel())
    states = [U]
    for _ in range(n_steps):
        U = lu.solve((1.0 - tau * r) * (ops.M @ U.ravel()) + src).reshape(q, q)
        states.append(U)
    return states


def imex_adjoint_src(ops, d_u, tau, r, states, dJ_dUN):
    """(dJ/dU_0, dJ/dd_u, dJ/dF (n x n), dJ/dr) of imex_forward_src by the adjoint
    recursion of the module docstring."""
    lu = ops.system(d_u, tau)
    q = ops.q
    n = int(round(np.sqrt(ops.M_all.shape[1])))
    lam = np.asarray(dJ_dUN, dtype=np.float64).ravel()
    g_du, g_r = 0.0, 0.0
    g_F = np.zeros(n * n)
    for i in range(len(states) - 2, -1, -1):
        y = lu.solve(lam)
        g_du -= tau * float(y @ (ops.A @ states[i + 1].ravel()))
        My = ops.M @ y          # M symmetric
        g_r -= tau * float(My @ states[i].ravel())
        g_F += tau * (ops.M_all.T @ y)
        lam = (1.0 - tau * r) * My
    return lam.reshape(q, q), g_du, g_F.reshape(n, n), g_r
