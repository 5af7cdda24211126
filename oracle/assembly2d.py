"""Vector-form 2D FEM assembly on the physical curvilinear mesh (oracle).

Test infrastructure only.

This is the "vector formulation" of the paper (Sec. 5, Eq. laplace_xnormal_FEM:
(A~ + gamma M~) xi = M~ f, and its lumped counterpart Eq.
laplace_xnormal_FEM_lumped).  It is written independently of the Kronecker
decomposition: every element integral is a 2D tensor quadrature on the
reference element, with the physical gradient obtained from the Jacobian of
the map eta(s, t) = (s, g1(s) + t h(s)) directly (Sec. 2.2, Eq. transformation
and the Jacobian J_eta) -- no H^ splitting, no weighted 1D matrices.  It exists
to pin :mod:`oracle.operator` on small grids.

Unknown ordering: node (a, b) -> a * n + b, i.e. row-major vec of U[a][b].
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fem1d import lagrange_ref, quadrature, interior


def assemble(problem):
    """Return (A + gamma M, M) as CSR matrices of size n^2 x n^2 (untrimmed)."""
    k = problem.k
    deg = 1 if k == 0 else k
    n = problem.n
    E = (n - 1) // deg
    hE = 1.0 / E
    xi, wq = quadrature(k, None if k == 0 else problem.mesh.xi.size)
    phi, dphi = lagrange_ref(deg, xi)
    nq = xi.size
    nl = deg + 1
    g1, dg1 = problem.g1.g, problem.g1.dg
    g2, dg2 = problem.g2.g, problem.g2.dg
    rows, cols, av, mv = [], [], [], []
    for es in range(E):
        s = (es + xi) * hE                      # (nq,)
        hs = g2(s) - g1(s)
        dhs = dg2(s) - dg1(s)
        d1 = dg1(s)
        for et in range(E):
            t = (et + xi) * hE
            # 2D quadrature points (qs, qt); local basis (a, b)
            # reference-derivatives scaled to (s, t): d/ds = dphi/hE
            # Jacobian of eta at (s, t): [[dx/ds, dx/dt], [dy/ds, dy/dt]]
            #   = [[1, 0], [g1' + t h', h]]
            Aloc = np.zeros((nl, nl, nl, nl))
            Mloc = np.zeros((nl, nl, nl, nl))
            for qs in range(nq):
                for qt in range(nq):
                    J = np.array([[1.0, 0.0], [d1[qs] + t[qt] * dhs[qs], hs[qs]]])
                    detJ = np.linalg.det(J)
                    JinvT = np.linalg.inv(J).T
                    wgt = wq[qs] * wq[qt] * hE * hE * abs(detJ)
                    # basis values and reference gradients for all (a, b)
                    val = np.outer(phi[:, qs], phi[:, qt])                  # (a, b)
                    gs = np.outer(dphi[:, qs] / hE, phi[:, qt])             # d/ds
                    gt = np.outer(phi[:, qs], dphi[:, qt] / hE)             # d/dt
                    # physical gradient: grad_xy = J^{-T} grad_st
                    gx = JinvT[0, 0] * gs + JinvT[0, 1] * gt
                    gy = JinvT[1, 0] * gs + JinvT[1, 1] * gt
                    Aloc += wgt * (np.einsum('ab,cd->abcd', gx, gx) + np.einsum('ab,cd->abcd', gy, gy))
                    Mloc += wgt * np.einsum('ab,cd->abcd', val, val)
            ga = es * deg + np.arange(nl)
            gb = et * deg + np.arange(nl)
            gid = (ga[:, None] * n + gb[None, :])                            # (a, b)
            I = np.broadcast_to(gid[:, :, None, None], Aloc.shape).ravel()
            Jc = np.broadcast_to(gid[None, None, :, :], Aloc.shape).ravel()
            rows.append(I)
            cols.append(Jc)
            av.append(Aloc.ravel())
            mv.append(Mloc.ravel())
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    A = sp.coo_matrix((np.concatenate(av), (rows, cols)), shape=(n * n, n * n)).tocsr()
    M = sp.coo_matrix((np.concatenate(mv), (rows, cols)), shape=(n * n, n * n)).tocsr()
    return (A + problem.gamma * M).tocsr(), M


def interior_ids(problem):
    i = interior(problem.n, problem.bc)
    return (i[:, None] * problem.n + i[None, :]).ravel()


def system(problem):
    """Trimmed system matrix (q^2 x q^2) and the rhs map (q^2 x n^2)."""
    K, M = assemble(problem)
    ii = interior_ids(problem)
    return K[ii][:, ii].tocsr(), M[ii].tocsr()


def direct_solve(problem, F):
    """Solve the vector-form system directly (sparse LU); returns U (q x q)."""
    K, Mr = system(problem)
    b = Mr @ np.asarray(F, dtype=np.float64).ravel()
    x = spla.spsolve(K.tocsc(), b)
    return x.reshape(problem.q, problem.q)
