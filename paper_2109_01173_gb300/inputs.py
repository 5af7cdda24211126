"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module only *describes workloads*: domain profiles, nodal right-hand
sides and seeded noise.  It holds none of the solver's arithmetic (no FEM
matrices, no operator, no preconditioner) and imports neither the CUDA binding
nor the oracle, so both sides can be fed the same arrays.

Workloads (all on x-normal domains {0 <= x <= 1, g1(x) <= y <= g2(x)}):

* ``config_p1_65``: -Lap u + u = f on g1 = 0, g2 = 1 + 0.25 sin(2 pi x), P1,
  65 x 65 nodes, zero Dirichlet data; f manufactured from
  u = sin(pi x) sin(pi y / g2(x)) plus seeded N(0, sigma = 1e-3) noise.
* ``fourier_f``: f = sum_j a_j / (1 + |m_j|^2) cos(2 pi (m_j . (x, y)) + phi_j) with
  32 modes, a_j ~ N(0, 1), m_j uniform in {-8..8}^2 \\ {0}, phi_j ~ U[0, 2 pi).
* ``batch_instances``: gamma ~ U[0, 10], g2 = 1 + a sin(2 pi b x) with
  a ~ U[0, 0.3], b in {1, 2, 3}, seeded per instance.
"""
import math
import numpy as np


class Profile:
    """g(x) = c0 + c1 x + c2 x^2 + sa sin(2 pi sf x) + ca cos(pi cf x), with g', g''."""

    def __init__(self, c0=0.0, c1=0.0, c2=0.0, sa=0.0, sf=1.0, ca=0.0, cf=1.0):
        self.c0, self.c1, self.c2 = float(c0), float(c1), float(c2)
        self.sa, self.sf, self.ca, self.cf = float(sa), float(sf), float(ca), float(cf)

    def g(self, x):
        x = np.asarray(x, dtype=np.float64)
        return (self.c0 + self.c1 * x + self.c2 * x * x
                + self.sa * np.sin(2 * np.pi * self.sf * x) + self.ca * np.cos(np.pi * self.cf * x))

    def dg(self, x):
        x = np.asarray(x, dtype=np.float64)
        w1, w2 = 2 * np.pi * self.sf, np.pi * self.cf
        return (self.c1 + 2 * self.c2 * x + self.sa * w1 * np.cos(w1 * x)
                - self.ca * w2 * np.sin(w2 * x))

    def d2g(self, x):
        x = np.asarray(x, dtype=np.float64)
        w1, w2 = 2 * np.pi * self.sf, np.pi * self.cf
        return (2 * self.c2 - self.sa * w1 * w1 * np.sin(w1 * x)
                - self.ca * w2 * w2 * np.cos(w2 * x))

    def is_zero(self):
        return self.c0 == 0 and self.c1 == 0 and self.c2 == 0 and self.sa == 0 and self.ca == 0

    def __repr__(self):
        return (f"Profile(c0={self.c0}, c1={self.c1}, c2={self.c2}, sa={self.sa}, sf={self.sf}, "
                f"ca={self.ca}, cf={self.cf})")


ZERO = Profile()
SIN_TOP = Profile(c0=1.0, sa=0.25, sf=1.0)           # 1 + 0.25 sin(2 pi x)


def nodal_xy(g1, g2, n):
    """Physical coordinates of the n x n mapped nodes: x = s_a, y = g1(s_a) + t_b h(s_a)."""
    s = np.arange(n, dtype=np.float64) / (n - 1)
    t = s.copy()
    lo, hi = g1.g(s), g2.g(s)
    X = np.repeat(s[:, None], n, axis=1)
    Y = lo[:, None] + t[None, :] * (hi - lo)[:, None]
    return X, Y


def manufactured_sin_f(g1, g2, n, gamma):
    """Nodal f = -Lap u + gamma u for u = sin(pi s) sin(pi t), t = (y - g1(x)) / h(x).

    u vanishes on the whole boundary of the domain.  Derivatives in physical
    coordinates: t_x = -(g1' + t h')/h, t_xx = -(g1'' + 2 t_x h' + t h'')/h,
    t_y = 1/h, t_yy = 0.
    """
    s = np.arange(n, dtype=np.float64) / (n - 1)
    S = np.repeat(s[:, None], n, axis=1)
    T = np.repeat(s[None, :], n, axis=0)
    h = (g2.g(s) - g1.g(s))[:, None]
    dh = (g2.dg(s) - g1.dg(s))[:, None]
    d2h = (g2.d2g(s) - g1.d2g(s))[:, None]
    d1, dd1 = g1.dg(s)[:, None], g1.d2g(s)[:, None]
    tx = -(d1 + T * dh) / h
    txx = -(dd1 + 2 * tx * dh + T * d2h) / h
    ty = 1.0 / h
    pi = np.pi
    ss, cs = np.sin(pi * S), np.cos(pi * S)
    st, ct = np.sin(pi * T), np.cos(pi * T)
    u = ss * st
    uxx = (-pi * pi * ss * st + 2 * pi * pi * cs * ct * tx - pi * pi * ss * st * tx * tx
           + pi * ss * ct * txx)
    uyy = -pi * pi * ss * st * ty * ty
    return -(uxx + uyy) + gamma * u, u


def _fourier_modes(seed, modes, mmax):
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.standard_normal(modes)
    m = np.zeros((modes, 2), dtype=np.int64)
    for j in range(modes):
        while True:
            cand = rng.integers(-mmax, mmax + 1, size=2)
            if cand[0] != 0 or cand[1] != 0:
                m[j] = cand
                break
    phi = rng.uniform(0.0, 2 * np.pi, size=modes)
    return a, m, phi


def fourier_f(g1, g2, n, seed, modes=32, mmax=8):
    """Seeded sum of random Fourier modes evaluated at the physical nodes."""
    a, m, phi = _fourier_modes(seed, modes, mmax)
    X, Y = nodal_xy(g1, g2, n)
    F = np.zeros((n, n))
    for j in range(modes):
        F += a[j] / (1.0 + float(m[j] @ m[j])) * np.cos(2 * np.pi * (m[j, 0] * X + m[j, 1] * Y) + phi[j])
    return F


def fourier_f_device(g1, g2, n, seed, device, modes=32, mmax=8):
    """fourier_f evaluated with torch in FP64 on `device` (the same modes and nodes; the
    cosines of the device library may differ from numpy's in the last bit): for large
    workloads whose right-hand sides only the GPU path reads."""
    import torch
    a, m, phi = _fourier_modes(seed, modes, mmax)
    X, Y = nodal_xy(g1, g2, n)
    Xd = torch.tensor(X, dtype=torch.float64, device=device)
    Yd = torch.tensor(Y, dtype=torch.float64, device=device)
    F = torch.zeros((n, n), dtype=torch.float64, device=device)
    for j in range(modes):
        F += float(a[j] / (1.0 + float(m[j] @ m[j]))) * torch.cos(
            2 * np.pi * (float(m[j, 0]) * Xd + float(m[j, 1]) * Yd) + float(phi[j]))
    return F


def noise(n, seed, sigma):
    rng = np.random.Generator(np.random.PCG64(seed))
    return sigma * rng.standard_normal((n, n))


def config_p1_65(seed=0):
    """P1, 65 x 65 nodes, gamma = 1, Dirichlet; manufactured f plus N(0, 1e-3) noise."""
    n, gamma = 65, 1.0
    f, u = manufactured_sin_f(ZERO, SIN_TOP, n, gamma)
    return dict(g1=ZERO, g2=SIN_TOP, k=1, n=n, gamma=gamma, bc='dirichlet',
                F=f + noise(n, seed, 1e-3), u_exact=u)


def metric_instance(n=2049, k=2, seed=0, gamma=1.0):
    """gamma = 1, g2 = 1 + 0.25 sin(2 pi x), Dirichlet, seeded 32-mode Fourier f."""
    return dict(g1=ZERO, g2=SIN_TOP, k=k, n=n, gamma=gamma, bc='dirichlet',
                F=fourier_f(ZERO, SIN_TOP, n, seed))


def batch_instances(B, n=2049, k=2, seed0=0, with_f=True):
    """B instances at fixed (n, k): gamma ~ U[0,10], g2 = 1 + a sin(2 pi b x), f seeded
    (with_f = False: only its seed, "f_seed", for fourier_f_device)."""
    out = []
    for i in range(B):
        rng = np.random.Generator(np.random.PCG64(1000 + seed0 + i))
        gamma = float(rng.uniform(0.0, 10.0))
        a = float(rng.uniform(0.0, 0.3))
        b = int(rng.integers(1, 4))
        g2 = Profile(c0=1.0, sa=a, sf=b)
        out.append(dict(g1=ZERO, g2=g2, k=k, n=n, gamma=gamma, bc='dirichlet', f_seed=seed0 + i,
                        F=fourier_f(ZERO, g2, n, seed0 + i) if with_f else None))
    return out


def smoothed_uniform(q, seed, sweeps=5, batch=None):
    """Seeded uniform[0, 1] field on q x q nodes smoothed by `sweeps` Jacobi sweeps.

    One sweep of weighted Jacobi (weight 2/3) for the 5-point Laplacian with zero
    right-hand side and reflecting edges: U <- U + (2/3) (mean of the 4 neighbours - U).
    The initial condition of the heat-equation differentiation workload.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (q, q) if batch is None else (batch, q, q)
    U = rng.uniform(0.0, 1.0, shape)
    for _ in range(sweeps):
        P = np.pad(U, [(0, 0)] * (U.ndim - 2) + [(1, 1), (1, 1)], mode="reflect")
        nb = 0.25 * (P[..., :-2, 1:-1] + P[..., 2:, 1:-1] + P[..., 1:-1, :-2] + P[..., 1:-1, 2:])
        U = U + (2.0 / 3.0) * (nb - U)
    return U


def heat_config():
    """Differentiation workload: u_t - d_u Lap u = 0, homogeneous Neumann BC, domain
    {0 <= x <= 1, 0.1 x^2 <= y <= 1 + 0.2 cos(pi x)}, P2 with 513 nodes per direction,
    IMEX Euler dt = 1e-3 for 400 steps, d_u = 0.05, checkpoints every 50 steps."""
    return dict(g1=Profile(c2=0.1), g2=Profile(c0=1.0, ca=0.2, cf=1.0), k=2, n=513, bc="neumann",
                d_u=0.05, tau=1e-3, steps=400, every=50)


def dib_params_cap():
    """DIB kinetics parameters: Eq. dib_parameters_mixed with the cap-domain A2, B, C (Sec. 7.1)."""
    return dict(alpha=0.5, gamma=0.2, A1=10.0, A2=30.0, B=25.0, C=7.0, D=3.2727, k2=2.5, k3=1.5, d_theta=20.0)


def dib_initial(n, eta_e, theta_e, seed=0, amplitude=1e-3):
    """[eta0; theta0] on n x n nodes: the given homogeneous state plus a seeded uniform
    perturbation in [-amplitude, amplitude] (initial data of the reaction-diffusion runs)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.stack([eta_e + rng.uniform(-amplitude, amplitude, (n, n)),
                     theta_e + rng.uniform(-amplitude, amplitude, (n, n))])


def hetero_instances(count, n_choices=(129, 257, 513, 1025, 2049), k_choices=(1, 2, 3, 4), seed=0, with_f=True):
    """Heterogeneous batch: per instance n ~ U(n_choices), k ~ U(k_choices) (n adjusted to
    3 floor((n-1)/3) + 1 when k = 3 does not divide n - 1), gamma ~ U[0, 10],
    g2 = 1 + a sin(2 pi b x) with a ~ U[0, 0.3], b ~ U{1, 2, 3}, Dirichlet, seeded
    32-mode Fourier f (with_f = False: only its seed, "f_seed", for fourier_f_device)."""
    rng = np.random.Generator(np.random.PCG64(5000 + seed))
    out = []
    for i in range(count):
        n = int(rng.choice(n_choices))
        k = int(rng.choice(k_choices))
        if (n - 1) % k:
            n = k * ((n - 1) // k) + 1
        gamma = float(rng.uniform(0.0, 10.0))
        g2 = Profile(c0=1.0, sa=float(rng.uniform(0.0, 0.3)), sf=int(rng.integers(1, 4)))
        fs = seed * 100000 + i
        out.append(dict(g1=ZERO, g2=g2, k=k, n=n, gamma=gamma, bc='dirichlet', f_seed=fs,
                        F=fourier_f(ZERO, g2, n, fs) if with_f else None))
    return out


CAP_LOWER = Profile(c0=-1.0, c2=0.5)     # y = x^2/2 - 1
CAP_UPPER = Profile(c0=1.0, c2=-0.5)     # y = 1 - x^2/2


def _poly_mul(a, b):
    """Product of two 2D coefficient arrays c[i, j] of x^i y^j."""
    out = np.zeros((a.shape[0] + b.shape[0] - 1, a.shape[1] + b.shape[1] - 1))
    for i in range(a.shape[0]):
        for j in range(a.shape[1]):
            out[i:i + b.shape[0], j:j + b.shape[1]] += a[i, j] * b
    return out


def cap_heat_problem(k, N, d_u=0.1):
    """The heat test on the cap-shaped domain (Sec. 6; x and y swapped to this
    orientation): x^2/2 - 1 <= y <= 1 - x^2/2, zero Dirichlet data,
    u(x, y, t) = u0(x, y) e^t with u0 = x (x - 1)(-x^2/2 + y + 1)(x^2/2 + y - 1), so
    f = e^t (u0 - d_u Lap u0).  N elements per direction of degree max(k, 1).
    Returns dict(g1, g2, k, n, d_u, u0 (n x n nodal), f(t) -> n x n nodal)."""
    P2 = np.polynomial.polynomial
    c = _poly_mul(_poly_mul(np.array([[0.0], [-1.0], [1.0]]), np.array([[1.0, 1.0], [0.0, 0.0], [-0.5, 0.0]])),
                  np.array([[-1.0, 1.0], [0.0, 0.0], [0.5, 0.0]]))
    lap = (np.pad(P2.polyder(c, 2, axis=0), ((0, 2), (0, 0))) +
           np.pad(P2.polyder(c, 2, axis=1), ((0, 0), (0, 2))))
    n = max(k, 1) * N + 1
    X, Y = nodal_xy(CAP_LOWER, CAP_UPPER, n)
    u0 = P2.polyval2d(X, Y, c)
    f0 = u0 - d_u * P2.polyval2d(X, Y, lap)
    return dict(g1=CAP_LOWER, g2=CAP_UPPER, k=k, n=n, d_u=d_u, u0=u0, f=lambda t: math.exp(t) * f0)
