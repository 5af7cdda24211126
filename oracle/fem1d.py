"""1D finite-element building blocks (oracle; test infrastructure only).

Sec. 2.1 (mesh K_h with equispaced nodes) and Sec. 3.1-3.3 of the paper:
the 1D stiffness and mass matrices (Eq. stiffness_mass_1D), the weighted 1D
matrices B1, B2, C1, C2, M1, M2, M3 (Eqs. newmatrix_1 .. newmatrix_7) and the
lumped P1 matrices built with the element-wise interpolant I_h (Sec. 3.3).

Conventions used throughout the oracle:

* ``n`` is the number of nodes per direction; degree-k Lagrange elements on
  ``E = (n-1)/k`` equal elements of [0, 1]; node ``m`` sits at ``m/(n-1)``.
* ``k = 0`` denotes lumped P1: P1 elements whose 1D integrals are all taken of
  the element-wise linear interpolant I_h of the integrand, i.e. with the
  two-point trapezoid rule on every element (reading of Sec. 3.3).
* P_k (k >= 1) integrals use Gauss-Legendre with ``nq`` points per element
  (default k + 3), which is exact for the polynomial weights 1, t, t^2.

Three weighted matrix kinds are built for a weight function w:

    K[w]_ij = int psi_i' psi_j' w       (stiffness-like, symmetric)
    M[w]_ij = int psi_i  psi_j  w       (mass-like, symmetric)
    G[w]_ij = int psi_i' psi_j  w       (convection-like; first index differentiated)

The paper's B1 = K[L], B2 = K[x^2], C1 = G[x], C2 = G[L'], M1 = M[1/L],
M2 = M[L'^2/L], M3 = M[L].
"""
import numpy as np
import scipy.sparse as sp


def lagrange_ref(k, xi):
    """Values and derivatives of the k+1 Lagrange polynomials on [0, 1].

    Nodes are xi_j = j/k (equispaced, Sec. 3.1 "piecewise Lagrange polynomials
    of any fixed degree").  Returns (phi, dphi), each of shape (k+1, len(xi)),
    with derivatives taken with respect to the reference coordinate xi.
    """
    xi = np.asarray(xi, dtype=np.float64)
    nodes = np.arange(k + 1, dtype=np.float64) / k
    phi = np.ones((k + 1, xi.size))
    dphi = np.zeros((k + 1, xi.size))
    for j in range(k + 1):
        others = [m for m in range(k + 1) if m != j]
        denom = np.prod([nodes[j] - nodes[m] for m in others])
        for m in others:
            phi[j] *= (xi - nodes[m])
        phi[j] /= denom
        # product rule: d/dxi prod_m (xi - x_m) = sum_l prod_{m != l} (xi - x_m)
        for l in others:
            term = np.ones(xi.size)
            for m in others:
                if m != l:
                    term *= (xi - nodes[m])
            dphi[j] += term
        dphi[j] /= denom
    return phi, dphi


def quadrature(k, nq=None):
    """Reference-element rule on [0, 1] (points, weights).

    P_k: Gauss-Legendre with nq points (default k + 3).  Lumped P1 (k = 0): the
    trapezoid rule, i.e. exact integration of the element-wise linear
    interpolant I_h of the integrand (Sec. 3.3).
    """
    if k == 0:
        return np.array([0.0, 1.0]), np.array([0.5, 0.5])
    if nq is None:
        nq = k + 3
    x, w = np.polynomial.legendre.leggauss(nq)
    return 0.5 * (x + 1.0), 0.5 * w


class Mesh1D:
    """Equispaced 1D mesh of degree-k elements with its quadrature data."""

    def __init__(self, n, k, nq=None):
        deg = 1 if k == 0 else k
        if n < 2 or (n - 1) % deg != 0:
            raise ValueError(f"n={n} nodes is not compatible with degree {deg}")
        self.n, self.k, self.deg = n, k, deg
        self.E = (n - 1) // deg
        self.h = 1.0 / self.E
        self.xi, self.wq = quadrature(k, nq)
        self.phi, self.dphi = lagrange_ref(deg, self.xi)   # (deg+1, nq)
        # physical quadrature points per element: (E, nq)
        e = np.arange(self.E, dtype=np.float64)[:, None]
        self.xq = (e + self.xi[None, :]) * self.h
        self.nodes = np.arange(n, dtype=np.float64) / (n - 1)

    def matrix(self, kind, weight):
        """Assemble K[w], M[w] or G[w] (kind 'K', 'M', 'G') as CSR (n x n).

        ``weight`` is a callable evaluated at the physical quadrature points,
        or None for w = 1.
        """
        w = np.ones_like(self.xq) if weight is None else np.asarray(weight(self.xq), dtype=np.float64)
        if w.shape != self.xq.shape:
            w = np.broadcast_to(w, self.xq.shape)
        d = self.dphi / self.h            # d psi / dx on the element
        v = self.phi
        if kind == 'K':
            left, right = d, d
        elif kind == 'M':
            left, right = v, v
        elif kind == 'G':
            left, right = d, v
        else:
            raise ValueError(kind)
        # local[e, a, c] = sum_q wq * h * w[e,q] * left[a,q] * right[c,q]
        local = np.einsum('q,eq,aq,cq->eac', self.wq * self.h, w, left, right)
        deg = self.deg
        rows, cols, vals = [], [], []
        for a in range(deg + 1):
            for c in range(deg + 1):
                rows.append(np.arange(self.E) * deg + a)
                cols.append(np.arange(self.E) * deg + c)
                vals.append(local[:, a, c])
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.n, self.n))
        return A.tocsr()


def interior(n, bc):
    """Indices kept after boundary trimming (Remark on Dirichlet BC, Eq. variable_dimension)."""
    if bc == 'dirichlet':
        return np.arange(1, n - 1)
    if bc == 'neumann':
        return np.arange(n)
    raise ValueError(bc)


def trim(A, rows, cols=None):
    """Remove boundary rows/columns (Dirichlet) from a CSR matrix."""
    if cols is None:
        cols = rows
    return A[rows][:, cols].tocsr()
