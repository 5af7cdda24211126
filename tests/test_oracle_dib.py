"""Pins of the DIB oracle (kinetics, equilibrium, coupled IMEX Euler) on the CPU.

* Kinetics: with C = 4 the pair (0, 1/2) zeroes f and g (D printed to 4 decimals,
  so g(0, 1/2) = 4 * 0.45 - 3.2727 * 0.55 = 1.5e-5); the hand-written Jacobian
  equals central differences of f and g.
* Kinetics at the points where the printed formulas collapse (theta = 0 and 1,
  eta = 0, the odd part in eta): every factor (k2, k3, the gamma brackets, A1, A2,
  B, alpha) sits where Sec. 7 prints it.
* Equilibrium: Newton's answer zeroes the kinetics (cap and jar parameters) and,
  for the cap parameters, equals the value obtained without the oracle.
* Lumped P1 with Neumann BC: the cosine vectors cos(i pi j / N) satisfy
  A v = lam M v with lam = 2 N^2 (1 - cos(i pi / N)) (closed form).
* Coupled IMEX Euler: the homogeneous equilibrium is a fixed point (constants are
  in the kernel of the Neumann stiffness); a small separable cosine perturbation of
  the equilibrium on the unit square evolves by the 2 x 2 amplification matrix
  G = diag(1 + tau lam, 1 + d_theta tau lam)^-1 (I + tau rho J) per step.
"""
import json
import os

import numpy as np
import pytest

from oracle import dib
from oracle.heat import HeatOperators
from oracle.fem1d import Mesh1D, interior
from paper_2109_01173_gb300.inputs import Profile, ZERO

ONE = Profile(c0=1.0)


def test_kinetics_zero_at_printed_equilibrium_for_c4():
    p = dict(dib.CAP, C=4.0)
    assert abs(dib.f(0.0, 0.5, p)) == 0.0
    assert abs(dib.g(0.0, 0.5, p)) <= 2e-5


@pytest.mark.parametrize("params", [dib.CAP, dib.JAR])
def test_jacobian_and_equilibrium(params):
    rng = np.random.default_rng(0)
    for _ in range(5):
        e, t = rng.uniform(-0.5, 0.5), rng.uniform(0.1, 0.9)
        J = dib.jacobian(e, t, params)
        h = 1e-6
        fd = np.array([[(dib.f(e + h, t, params) - dib.f(e - h, t, params)) / (2 * h),
                        (dib.f(e, t + h, params) - dib.f(e, t - h, params)) / (2 * h)],
                       [(dib.g(e + h, t, params) - dib.g(e - h, t, params)) / (2 * h),
                        (dib.g(e, t + h, params) - dib.g(e, t - h, params)) / (2 * h)]])
        assert np.abs(J - fd).max() <= 1e-7 * max(1.0, np.abs(J).max())
    e, t = dib.equilibrium(params)
    assert abs(dib.f(e, t, params)) <= 1e-12 and abs(dib.g(e, t, params)) <= 1e-12


def test_lumped_neumann_cosine_eigenpairs():
    N = 12
    m = Mesh1D(N + 1, 0)
    idx = interior(N + 1, 'neumann')
    A = m.matrix('K', None).toarray()[np.ix_(idx, idx)]
    M = m.matrix('M', None).toarray()[np.ix_(idx, idx)]
    j = np.arange(N + 1)
    for i in range(N + 1):
        v = np.cos(i * np.pi * j / N)
        lam = 2.0 * N * N * (1.0 - np.cos(i * np.pi / N))
        assert np.abs(A @ v - lam * (M @ v)).max() <= 1e-10 * max(1.0, lam)


def test_equilibrium_is_a_fixed_point_of_imex():
    p = dib.CAP
    ops = HeatOperators(ZERO, Profile(c0=1.0, sa=0.25), 0, 9, 'neumann')
    e, t = dib.equilibrium(p)
    q = ops.q
    eta, theta, _ = dib.imex(ops, p, 1.0, 1e-2, np.full((q, q), e), np.full((q, q), t), 20)
    assert np.abs(eta - e).max() <= 1e-13 and np.abs(theta - t).max() <= 1e-13


def test_small_cosine_mode_follows_the_amplification_matrix():
    p, rho, tau, steps, N = dib.CAP, 1.0, 1e-2, 10, 10
    ops = HeatOperators(ZERO, ONE, 0, N + 1, 'neumann')
    e, t = dib.equilibrium(p)
    j = np.arange(N + 1)
    i1, i2 = 1, 0
    mode = np.outer(np.cos(i1 * np.pi * j / N), np.cos(i2 * np.pi * j / N))
    lam = 2 * N * N * ((1 - np.cos(i1 * np.pi / N)) + (1 - np.cos(i2 * np.pi / N)))
    a0 = np.array([1e-7, -2e-7])   # nonlinear terms O(a^2): ~1e-6 of the mode after 10 steps
    eta, theta, _ = dib.imex(ops, p, rho, tau, e + a0[0] * mode, t + a0[1] * mode, steps)
    G = np.linalg.solve(np.diag([1 + tau * lam, 1 + p['d_theta'] * tau * lam]),
                        np.eye(2) + tau * rho * dib.jacobian(e, t, p))
    a = np.linalg.matrix_power(G, steps) @ a0
    assert np.abs((eta - e) - a[0] * mode).max() <= 1e-5 * np.abs(a).max()
    assert np.abs((theta - t) - a[1] * mode).max() <= 1e-5 * np.abs(a).max()


GOLD_IND = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "independent_values.json")))


@pytest.mark.parametrize("params", [dib.CAP, dib.JAR])
def test_kinetics_special_cases_place_every_factor(params):
    """Sec. 7, Eqs. dib_kinetics_f and dib_kinetics_g at the points where they collapse:
    theta = 1 leaves only the D-term of g, -D (1 + gamma)(1 + k3 eta) (places k3 and the
    gamma theta factor); theta = 0 leaves only the C-term, C (1 - gamma)(1 + k2 eta)
    (places k2 and the bracket); g is affine in eta; f(0, theta) = -B (theta - alpha),
    f - f(0, .) is odd in eta with cubic coefficient -A2 and linear coefficient
    A1 (1 - theta)."""
    p = params
    for eta in (-0.7, -0.2, 0.0, 0.3, 1.1):
        assert dib.g(eta, 1.0, p) == pytest.approx(-p['D'] * (1 + p['gamma']) * (1 + p['k3'] * eta), rel=1e-14, abs=1e-14)
        assert dib.g(eta, 0.0, p) == pytest.approx(p['C'] * (1 - p['gamma']) * (1 + p['k2'] * eta), rel=1e-14, abs=1e-14)
    for theta in (0.1, 0.5, 0.8):
        g = [dib.g(e, theta, p) for e in (-1.0, 0.0, 1.0)]
        assert abs(g[0] - 2 * g[1] + g[2]) <= 1e-12 * max(1.0, abs(g[1]))
        assert dib.f(0.0, theta, p) == pytest.approx(-p['B'] * (theta - p['alpha']), rel=1e-14, abs=1e-14)
        odd = [(dib.f(e, theta, p) - dib.f(-e, theta, p)) / 2 for e in (0.5, 1.0)]
        # odd part c1 e + c3 e^3 from two samples
        c3 = (odd[1] - 2 * odd[0]) / (1.0 - 2 * 0.125)
        c1 = odd[1] - c3
        assert c3 == pytest.approx(-p['A2'], rel=1e-12)
        assert c1 == pytest.approx(p['A1'] * (1 - theta), rel=1e-12)


def test_cap_equilibrium_matches_the_independent_value():
    """Newton's zero of the oracle kinetics with the printed cap parameters equals the
    value obtained without the oracle (elimination of eta from g = 0, bisection in theta;
    tests/golden/independent_values.json), to its 4 digits."""
    e, t = dib.equilibrium(dib.CAP)
    want = GOLD_IND["dib_cap_equilibrium"]
    assert abs(e - want["eta"]) <= 0.6e-4 and abs(t - want["theta"]) <= 0.6e-4, (e, t)
