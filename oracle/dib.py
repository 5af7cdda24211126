"""DIB reaction-diffusion model and its IMEX Euler integration (oracle).

Test infrastructure only: only tests/, the package's smoke check and the bench's
CPU baseline may import it.

Sec. 7, Eqs. dib_model, dib_kinetics_f, dib_kinetics_g: with zero Neumann data

    eta_t   -         Lap eta   = rho f(eta, theta),
    theta_t - d_theta Lap theta = rho g(eta, theta),
    f = A1 (1 - theta) eta - A2 eta^3 - B (theta - alpha),
    g = C (1 + k2 eta)(1 - theta)[1 - gamma (1 - theta)] - D theta (1 + gamma theta)(1 + k3 eta),

with the parameters of Eq. dib_parameters_mixed (alpha, gamma, A1, D, k2, k3,
d_theta) and the per-domain (A2, B, C) of Sec. 7.1 (cap) and 7.2 (jar).

IMEX Euler as in Sec. 6: diffusion implicit, reaction explicit, each species
its own sparse direct solve (M~ + d tau A~) U_{n+1} = M~ (U_n + tau rho F(U_n))
with the operators of oracle/heat.py.

Reading (the paper is inconsistent here): with the printed D = 3.2727 the pair
(0, 0.5) is a zero of the kinetics only for C = 4 (g(0, 1/2) = C 0.45 - D 0.55);
with the printed C = 7 (cap) or 3 (jar) the homogeneous equilibrium is computed
by Newton's method from (0, 0.5).
"""
import numpy as np

from .heat import HeatOperators

BASE = dict(alpha=0.5, gamma=0.2, A1=10.0, D=3.2727, k2=2.5, k3=1.5, d_theta=20.0)
CAP = dict(BASE, A2=30.0, B=25.0, C=7.0)
JAR = dict(BASE, A2=1.0, B=30.0, C=3.0)


def f(eta, theta, p):
    return p['A1'] * (1.0 - theta) * eta - p['A2'] * eta ** 3 - p['B'] * (theta - p['alpha'])


def g(eta, theta, p):
    return (p['C'] * (1.0 + p['k2'] * eta) * (1.0 - theta) * (1.0 - p['gamma'] * (1.0 - theta))
            - p['D'] * theta * (1.0 + p['gamma'] * theta) * (1.0 + p['k3'] * eta))


def jacobian(eta, theta, p):
    """[[f_eta, f_theta], [g_eta, g_theta]] by differentiating the kinetics by hand."""
    ga = p['gamma']
    f_e = p['A1'] * (1.0 - theta) - 3.0 * p['A2'] * eta ** 2
    f_t = -p['A1'] * eta - p['B']
    w = (1.0 - theta) * (1.0 - ga * (1.0 - theta))          # C-part without (1 + k2 eta)
    dw = -(1.0 - ga * (1.0 - theta)) + (1.0 - theta) * ga   # d w / d theta
    v = theta * (1.0 + ga * theta)                          # D-part without (1 + k3 eta)
    dv = 1.0 + 2.0 * ga * theta
    g_e = p['C'] * p['k2'] * w - p['D'] * v * p['k3']
    g_t = p['C'] * (1.0 + p['k2'] * eta) * dw - p['D'] * dv * (1.0 + p['k3'] * eta)
    return np.array([[f_e, f_t], [g_e, g_t]])


def equilibrium(p, guess=(0.0, 0.5), tol=1e-15, max_iter=50):
    """Homogeneous equilibrium (f = g = 0) by Newton's method."""
    x = np.array(guess, dtype=np.float64)
    for _ in range(max_iter):
        r = np.array([f(x[0], x[1], p), g(x[0], x[1], p)])
        dx = np.linalg.solve(jacobian(x[0], x[1], p), r)
        x = x - dx
        if np.abs(dx).max() <= tol * max(1.0, np.abs(x).max()):
            break
    return float(x[0]), float(x[1])


def imex(ops, p, rho, tau, eta0, theta0, n_steps, record_every=0):
    """(eta_N, theta_N, records): IMEX Euler; records = [(n, eta_n, theta_n)] every record_every steps."""
    lu_e = ops.system(1.0, tau)
    lu_t = ops.system(p['d_theta'], tau)
    q = ops.q
    eta = np.asarray(eta0, dtype=np.float64).reshape(q, q)
    theta = np.asarray(theta0, dtype=np.float64).reshape(q, q)
    rec = []
    for n in range(n_steps):
        fe = rho * f(eta, theta, p)
        ft = rho * g(eta, theta, p)
        eta_new = lu_e.solve(ops.M @ (eta + tau * fe).ravel()).reshape(q, q)
        theta = lu_t.solve(ops.M @ (theta + tau * ft).ravel()).reshape(q, q)
        eta = eta_new
        if record_every and (n + 1) % record_every == 0:
            rec.append((n + 1, eta.copy(), theta.copy()))
    return eta, theta, rec


def operators(g1, g2, n, k=0):
    """Neumann operators of the DIB runs (lumped P1 by default)."""
    return HeatOperators(g1, g2, k, n, 'neumann')
