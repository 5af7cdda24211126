"""Pins of the oracle's IMEX Euler heat solver and its discrete adjoint (CPU).

* Forward: on the unit square with P1 and Dirichlet BC a separable sine mode
  v_i v_j^T is an eigenvector of M~^{-1} A~ with eigenvalue lam_i + lam_j (the 1D
  eigenvalues of M^{-1} A, Sec. 4.1 with the corrected Eq. dirichlet_eigenvalues),
  so N steps multiply it by (1 + d tau (lam_i + lam_j))^{-N} exactly.
* d_u gradient: for that mode and J = ||U_N - c0 U_0||^2 the derivative is a
  closed form in d.
* Adjoint against the forward map: on curved two-profile domains (eight terms,
  Dirichlet and Neumann, P1/P2) the adjoint gradient equals central finite
  differences of the forward solve, for U_0 along random directions and for d_u;
  with a nodal source f and an explicit linear reaction r u, also for f along random
  nodal directions and for r.
* Source and reaction: with f = 0 the square's sine mode is multiplied by
  (1 - tau r) / (1 + d tau (lam_i + lam_j)) per step, so J and dJ/dr have a closed
  form; f = 0 and r = 0 reduce the extended recursion to the plain one.
* Convergence: the paper's heat test on the cap-shaped domain (Sec. 6, Test 1:
  d_u = 0.1, u = u(x, y, 0) e^t, the step shrinking by 2^(k+1) per mesh halving)
  reaches its printed rates (k + 1; lumped P1 and P1: 2) on two coarse meshes.  At
  these sizes the first-order time error dominates, so this pins the time stepping
  and its schedule more than the space discretisation (which the 2D assembly and the
  elliptic manufactured rates pin): a load without the boundary nodes' f still
  passes it.
* Iterations: with the paper's heat preconditioner and stopping rule (Sec. 6, Test 2)
  MO-PCG takes one iteration per step for P_k (at most two for lumped P1); the plain
  mass preconditioner that the paper improves on takes more.
"""
import json
import os

import numpy as np
import pytest

from oracle import closed_form
from oracle.heat import (HeatOperators, imex_forward, imex_adjoint, loss, paper_heat_preconditioner,
                         imex_mo_pcg_step, imex_forward_src, imex_adjoint_src)
from oracle.fem1d import trim
from oracle.pcg import ProductPreconditioner
from oracle.operator import Problem
from oracle.operator import rhs
from paper_2109_01173_gb300.inputs import Profile, ZERO

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_printed_values.json")))

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


def _pmul(a, b):
    out = np.zeros((a.shape[0] + b.shape[0] - 1, a.shape[1] + b.shape[1] - 1))
    for i in range(a.shape[0]):
        for j in range(a.shape[1]):
            out[i:i + b.shape[0], j:j + b.shape[1]] += a[i, j] * b
    return out


def _cap_heat_error(k, N, tau):
    """Nodal RMS error at t = 1 of IMEX Euler on the paper's cap-domain heat problem
    (Sec. 6, Test 1), written in this orientation (x <-> y swapped): domain
    x^2/2 - 1 <= y <= 1 - x^2/2, u0 = x (x - 1) (-x^2/2 + y + 1) (x^2/2 + y - 1),
    u = u0 e^t, so f = e^t (u0 - d_u Lap u0).  Each step solves
    (M~ + d_u tau A~) U_{n+1} = M~ U_n + tau M_{int,all} f(t_n): the load is the mass of
    the interior test functions against the nodal f on all nodes (f does not vanish on
    the boundary)."""
    P2 = np.polynomial.polynomial
    c = _pmul(_pmul(np.array([[0.0], [-1.0], [1.0]]), np.array([[1.0, 1.0], [0.0, 0.0], [-0.5, 0.0]])),
              np.array([[-1.0, 1.0], [0.0, 0.0], [0.5, 0.0]]))
    lap = np.pad(P2.polyder(c, 2, axis=0), ((0, 2), (0, 0))) + np.pad(P2.polyder(c, 2, axis=1), ((0, 0), (0, 2)))
    g1, g2 = Profile(c0=-1.0, c2=0.5), Profile(c0=1.0, c2=-0.5)
    d_u = 0.1
    n = max(k, 1) * N + 1
    ops = HeatOperators(g1, g2, k, n)
    s = np.arange(n) / (n - 1)
    X = np.repeat(s[:, None], n, 1)
    Y = g1.g(s)[:, None] + s[None, :] * (g2.g(s) - g1.g(s))[:, None]
    u0 = P2.polyval2d(X, Y, c)
    l0 = P2.polyval2d(X, Y, lap)
    lu = ops.system(d_u, tau)
    U = u0[1:-1, 1:-1].copy()
    for st in range(int(round(1.0 / tau))):
        b = ops.M @ U.ravel() + tau * rhs(ops.problem, np.exp(st * tau) * (u0 - d_u * l0)).ravel()
        U = lu.solve(b).reshape(U.shape)
    err = U - np.e * u0[1:-1, 1:-1]
    return float(np.sqrt(np.mean(err ** 2)))


@pytest.mark.parametrize("k,name,N", [(0, "lumped_p1", 12), (1, "p1", 12), (2, "p2", 6), (3, "p3", 4), (4, "p4", 3)])
def test_cap_heat_rates_match_the_paper(k, name, N):
    """Two meshes N and 2N (elements per direction), steps 0.01 and 0.01 / 2^(k+1) (k = 1
    for lumped P1): the
    printed rates (Matrix PCG column) within 0.15.  The paper prints the step as
    0.01 * 2^((k+1)(i-1)); read with a negative exponent (the step shrinks as the mesh
    is refined, as its stated purpose, first order in time against order k+1 in space,
    requires)."""
    deg = max(k, 1)   # lumped P1 is of degree 1
    e1 = _cap_heat_error(k, N, 0.01)
    e2 = _cap_heat_error(k, 2 * N, 0.01 / 2 ** (deg + 1))
    r = np.log2(e1 / e2)
    want = GOLD["heat_cap_domain_rates_mo_pcg"]["value"][name]
    assert abs(r - want) <= 0.15, (k, r, want)


def _cap_heat_iterations(k, N, precond_kind, steps=10):
    """MO-PCG iterations of each of the first IMEX steps of the cap-domain heat test."""
    P2 = np.polynomial.polynomial
    c = _pmul(_pmul(np.array([[0.0], [-1.0], [1.0]]), np.array([[1.0, 1.0], [0.0, 0.0], [-0.5, 0.0]])),
              np.array([[-1.0, 1.0], [0.0, 0.0], [0.5, 0.0]]))
    lap = np.pad(P2.polyder(c, 2, axis=0), ((0, 2), (0, 0))) + np.pad(P2.polyder(c, 2, axis=1), ((0, 0), (0, 2)))
    g1, g2 = Profile(c0=-1.0, c2=0.5), Profile(c0=1.0, c2=-0.5)
    d_u, tau = 0.1, 0.01
    n = max(k, 1) * N + 1
    P = Problem(g1, g2, k, n, 0.0)
    if precond_kind == "paper":
        pre = paper_heat_preconditioner(P, d_u, tau)
    else:   # the plain mass preconditioner M3 U M
        f = P.factors()
        pre = ProductPreconditioner(trim(f['Ms_h'], P.idx).tocsr(), trim(f['Mt'], P.idx).tocsr())
    s = np.arange(n) / (n - 1)
    X = np.repeat(s[:, None], n, 1)
    Y = g1.g(s)[:, None] + s[None, :] * (g2.g(s) - g1.g(s))[:, None]
    u0 = P2.polyval2d(X, Y, c)
    l0 = P2.polyval2d(X, Y, lap)
    U = u0[1:-1, 1:-1].copy()
    its = []
    for st in range(steps):
        U, it = imex_mo_pcg_step(P, d_u, tau, U, np.exp(st * tau) * (u0 - d_u * l0), pre)
        its.append(it)
    return its


@pytest.mark.parametrize("k,N", [(1, 48), (2, 24), (3, 12), (4, 12)])
def test_paper_heat_preconditioner_one_iteration_per_step(k, N):
    its = _cap_heat_iterations(k, N, "paper")
    assert all(i == GOLD["heat_mo_pcg_iterations_per_step"]["value"]["p_k"] for i in its), its


def test_paper_heat_preconditioner_lumped_and_mass_only():
    its = _cap_heat_iterations(0, 48, "paper")
    assert max(its) <= GOLD["heat_mo_pcg_iterations_per_step"]["value"]["lumped_p1_at_most"], its
    # the uncorrected mass preconditioner the paper starts from needs more iterations
    assert max(_cap_heat_iterations(1, 48, "mass")) >= 3


def test_square_reaction_gradient_closed_form():
    N, d, tau, steps, c0, r = 12, 0.2, 0.02, 5, 0.5, 1.5
    ops = HeatOperators(ZERO, ONE, 1, N + 1, 'dirichlet')
    U0, Lam = _mode(N, 2, 1)
    F0 = np.zeros((N + 1, N + 1))
    states = imex_forward_src(ops, d, tau, U0, steps, F0, r)
    J, dJ = loss(states[-1], c0 * U0)
    _, g_du, g_F, g_r = imex_adjoint_src(ops, d, tau, r, states, dJ)
    g = (1.0 - tau * r) / (1.0 + d * tau * Lam)
    c = g ** steps
    dc_dr = steps * g ** (steps - 1) * (-tau) / (1.0 + d * tau * Lam)
    uu = float(np.sum(U0 * U0))
    assert abs(J - (c - c0) ** 2 * uu) <= 1e-12 * J
    assert abs(g_r - 2.0 * (c - c0) * dc_dr * uu) <= 1e-10 * abs(2.0 * (c - c0) * dc_dr * uu)
    dc_dd = steps * g ** (steps - 1) * (1.0 - tau * r) * (-tau * Lam) / (1.0 + d * tau * Lam) ** 2
    assert abs(g_du - 2.0 * (c - c0) * dc_dd * uu) <= 1e-10 * abs(2.0 * (c - c0) * dc_dd * uu)


def test_source_reaction_recursion_reduces_to_the_plain_one():
    ops = HeatOperators(G1, G2, 2, 9, 'neumann')
    q = ops.q
    rng = np.random.default_rng(4)
    U0, T = rng.uniform(0, 1, (q, q)), rng.uniform(0, 1, (q, q))
    st0 = imex_forward(ops, 0.05, 2e-2, U0, 4)
    st1 = imex_forward_src(ops, 0.05, 2e-2, U0, 4, np.zeros((9, 9)), 0.0)
    assert max(np.abs(a - b).max() for a, b in zip(st0, st1)) == 0.0
    dJ = loss(st0[-1], T)[1]
    g0 = imex_adjoint(ops, 0.05, 2e-2, st0, dJ)
    g1 = imex_adjoint_src(ops, 0.05, 2e-2, 0.0, st1, dJ)
    assert np.abs(g0[0] - g1[0]).max() <= 1e-14 * np.abs(g0[0]).max() and abs(g0[1] - g1[1]) <= 1e-14 * abs(g0[1])


@pytest.mark.parametrize("k,n,bc", [(1, 9, "dirichlet"), (2, 9, "neumann"), (0, 8, "dirichlet")])
def test_source_reaction_adjoint_equals_central_differences(k, n, bc):
    d, tau, steps, r = 0.05, 2e-2, 6, 0.7
    ops = HeatOperators(G1, G2, k, n, bc)
    q = ops.q
    rng = np.random.default_rng(7 * k + n)
    U0, T = rng.uniform(0, 1, (q, q)), rng.uniform(0, 1, (q, q))
    F = rng.standard_normal((n, n))

    def J_of(U=U0, dd=d, FF=F, rr=r):
        return loss(imex_forward_src(ops, dd, tau, U, steps, FF, rr)[-1], T)[0]

    states = imex_forward_src(ops, d, tau, U0, steps, F, r)
    dJ = loss(states[-1], T)[1]
    gU, g_du, g_F, g_r = imex_adjoint_src(ops, d, tau, r, states, dJ)
    for _ in range(2):   # J is quadratic in U_0 and in F: central differences exact up to rounding
        V = rng.standard_normal((q, q))
        fd = (J_of(U=U0 + 1e-3 * V) - J_of(U=U0 - 1e-3 * V)) / 2e-3
        assert abs(fd - float(np.sum(gU * V))) <= 1e-8 * abs(fd) + 1e-12
        W = rng.standard_normal((n, n))
        fd = (J_of(FF=F + 1e-3 * W) - J_of(FF=F - 1e-3 * W)) / 2e-3
        assert abs(fd - float(np.sum(g_F * W))) <= 1e-8 * abs(fd) + 1e-12
    for name, val, g in (("d_u", d, g_du), ("r", r, g_r)):
        eps = 1e-5 * val
        if name == "d_u":
            fd = (J_of(dd=d + eps) - J_of(dd=d - eps)) / (2 * eps)
        else:
            fd = (J_of(rr=r + eps) - J_of(rr=r - eps)) / (2 * eps)
        assert abs(fd - g) <= 1e-6 * abs(fd), (name, fd, g)
