"""Multiterm Sylvester operator of MO-FEM on a two-profile x-normal domain (oracle).

Test infrastructure only.

Geometry (Sec. 2.2, Eqs. transformation and hat-H, generalised to two
profiles as the Remark on symmetric / non-symmetric x-normal domains allows):
the domain is {0 <= x <= 1, g1(x) <= y <= g2(x)} and the map from the
reference square is (s, t) -> (x, y) = (s, g1(s) + t h(s)) with h = g2 - g1 > 0.
Its Jacobian determinant is h and the pulled-back diffusion tensor is

    H^ = [[ h , -w ], [ -w , (1 + w^2)/h ]],   w(s, t) = g1'(s) + t h'(s).

(With g1 = 0 and (s, t) = (paper y, paper x) this is the paper's Eq. hat-H.)

The unknown is the matrix U[a][b], a = s-node (row), b = t-node (column), and a
Kronecker term S (x) T acts as U -> S U T^T.  Expanding H^ into separable
pieces (Sec. 3.2, Eq. x-normal-decomposition-stiffness) gives eight terms

    (K_s[h] + gamma M_s[h])   (x) M_t
    M_s[(1 + g1'^2)/h]        (x) K_t[1]
    M_s[2 g1' h'/h]           (x) K_t[t]
    M_s[h'^2/h]               (x) K_t[t^2]
    -G_s[g1']                 (x) C_t[1]^T
    -G_s[g1']^T               (x) C_t[1]
    -G_s[h']                  (x) C_t[t]^T
    -G_s[h']^T                (x) C_t[t]

(C_t[w] is the G-kind matrix in t).  For g1' = 0 the third, fifth and sixth
vanish and the remaining five are the paper's Eq. kronecker_mass_distorted
(A (x) M1 + M (x) B1 + B2 (x) M2 - C1 (x) C2^T - C1^T (x) C2) plus gamma times the
mass M (x) M3, in the paper's index orientation.

The right-hand side is the mass matrix applied to the nodal values of f
(Sec. 4, Eq. poisson_square_FEM; Sec. 5, Eq. laplace_xnormal_FEM): with
Dirichlet trimming, interior test functions against the full nodal f.
"""
import numpy as np
import scipy.sparse as sp

from .fem1d import Mesh1D, interior, trim


class Profile:
    """A profile y = g(x) given by callables for g and g' (vectorised)."""

    def __init__(self, g, dg):
        self.g, self.dg = g, dg


class Problem:
    """-Lap u + gamma u = f on {0<=x<=1, g1(x)<=y<=g2(x)}, zero Dirichlet or Neumann BC.

    ``k`` in 1..4 for P_k, 0 for lumped P1.  ``n`` nodes per direction.
    """

    def __init__(self, g1, g2, k, n, gamma, bc='dirichlet', nq=None):
        self.g1, self.g2, self.k, self.n, self.gamma, self.bc = g1, g2, k, n, float(gamma), bc
        self.mesh = Mesh1D(n, k, nq)
        self.idx = interior(n, bc)
        self.q = self.idx.size

    # --- geometry (Sec. 2.2) -------------------------------------------------
    def h(self, s):
        return self.g2.g(s) - self.g1.g(s)

    def dh(self, s):
        return self.g2.dg(s) - self.g1.dg(s)

    # --- 1D factors (Sec. 3.2, Eqs. newmatrix_1 .. newmatrix_7, generalised) -
    def factors(self):
        """Untrimmed 1D factor matrices (n x n, CSR), keyed by name."""
        m = self.mesh
        h, dh, dg1 = self.h, self.dh, self.g1.dg
        f = {}
        f['Ks_h'] = m.matrix('K', h)
        f['Ms_h'] = m.matrix('M', h)
        f['Ms_a'] = m.matrix('M', lambda s: (1.0 + dg1(s) ** 2) / h(s))
        f['Ms_b'] = m.matrix('M', lambda s: 2.0 * dg1(s) * dh(s) / h(s))
        f['Ms_c'] = m.matrix('M', lambda s: dh(s) ** 2 / h(s))
        f['Gs_g1'] = m.matrix('G', dg1)
        f['Gs_dh'] = m.matrix('G', dh)
        f['Mt'] = m.matrix('M', None)
        f['Kt_1'] = m.matrix('K', None)
        f['Kt_t'] = m.matrix('K', lambda t: t)
        f['Kt_t2'] = m.matrix('K', lambda t: t * t)
        f['Ct_1'] = m.matrix('G', None)
        f['Ct_t'] = m.matrix('G', lambda t: t)
        return f

    def terms(self):
        """The eight (S_i, T_i) pairs, trimmed to q x q (CSR); zero terms are kept."""
        f = self.factors()
        i = self.idx
        tr = lambda A: trim(A, i)
        S1 = f['Ks_h'] + self.gamma * f['Ms_h']
        return [
            (tr(S1), tr(f['Mt'])),
            (tr(f['Ms_a']), tr(f['Kt_1'])),
            (tr(f['Ms_b']), tr(f['Kt_t'])),
            (tr(f['Ms_c']), tr(f['Kt_t2'])),
            (tr(-f['Gs_g1']), tr(f['Ct_1'].T.tocsr())),
            (tr(-f['Gs_g1'].T.tocsr()), tr(f['Ct_1'])),
            (tr(-f['Gs_dh']), tr(f['Ct_t'].T.tocsr())),
            (tr(-f['Gs_dh'].T.tocsr()), tr(f['Ct_t'])),
        ]

    def rhs_factors(self):
        """(M_s[h] rows=interior, cols=all ; M_t rows=interior, cols=all)."""
        f = self.factors()
        allc = np.arange(self.n)
        return trim(f['Ms_h'], self.idx, allc), trim(f['Mt'], self.idx, allc)

    def pencils(self, variant='averaged'):
        """Dense (E1, E2, F1, F2) of the two-term Sylvester preconditioner.

        E1 Z F1^T + E2 Z F2^T keeps the operator's two Kronecker terms whose
        t-factors are M_t and K_t: E1 = K_s[h] + gamma M_s[h], F1 = M_t, F2 = K_t,
        and E2 = M_s[e2] with
          'dominant':  e2 = (1 + g1'^2)/h                       (t-independent part)
          'averaged':  e2 = (1 + g1'^2 + g1' h' + h'^2/3)/h     (mean over t in [0,1]
                        of H^_tt = (1 + (g1' + t h')^2)/h, so the K_t[t], K_t[t^2]
                        terms enter with their t-averages)
        On the square (h = 1, g1 = 0) both equal the whole operator (Sec. 4, Eq.
        laplace_dirichlet_sylvester), so MO-PCG stops after one iteration.
        """
        t = self.terms()
        if variant == 'dominant':
            E2 = t[1][0]
        elif variant == 'averaged':
            h, dh, d1 = self.h, self.dh, self.g1.dg
            E2 = trim(self.mesh.matrix(
                'M', lambda s: (1.0 + d1(s) ** 2 + d1(s) * dh(s) + dh(s) ** 2 / 3.0) / h(s)), self.idx)
        else:
            raise ValueError(variant)
        return (t[0][0].toarray(), E2.toarray(), t[0][1].toarray(), t[1][1].toarray())

    def product_factors(self):
        """(E, F) of the paper's single-term preconditioner P(U) = E U F^T.

        Sec. 5, Eq. vector_preconditioner: P(U) = B1 U (A + B2), which in this
        orientation is K_s[h] U (K_t + K_t[t^2])^T.
        """
        f = self.factors()
        i = self.idx
        return trim(f['Ks_h'], i), trim(f['Kt_1'] + f['Kt_t2'], i)


def apply_terms(terms, U):
    """L(U) = sum_i S_i U T_i^T (Sec. 5, operator L~)."""
    Y = np.zeros_like(U, dtype=np.float64)
    for S, T in terms:
        Y += S @ (T @ U.T).T
    return Y


def rhs(problem, F):
    """B = M_s[h]_{int,all} F M_t_{int,all}^T for the nodal n x n field F (operator R~)."""
    Ms, Mt = problem.rhs_factors()
    return Ms @ (Mt @ np.asarray(F, dtype=np.float64).T).T


def apply_entry(terms_dense_rows, U, a, b):
    """One output entry L(U)[a, b] computed as an explicit double sum.

    ``terms_dense_rows`` is the list of (S, T) CSR pairs; only row a of S_i
    and row b of T_i are touched, so this stays cheap at any size and is used
    to check sampled outputs of large applies.
    """
    acc = 0.0
    for S, T in terms_dense_rows:
        srow = S.getrow(a)
        trow = T.getrow(b)
        for c, sv in zip(srow.indices, srow.data):
            for d, tv in zip(trow.indices, trow.data):
                acc += sv * tv * U[c, d]
    return acc
