"""GPU parity of the IMEX heat integration and its adjoint (differentiation form).

* Forward steps and adjoint gradients (dJ/dU_0, dJ/dd_u) against the FP64 oracle
  (sparse direct solves, oracle/heat.py) on small grids: Dirichlet and Neumann,
  P2 and lumped P1, the two-profile domain of the workload (eight terms).
* With a nodal source f and an explicit linear reaction -r u (u_t - d_u Lap u =
  f - r u): the states and all four gradients (U_0, d_u, f, r) against the oracle's
  extended adjoint on small grids.
* The workload itself (Neumann, 0.1 x^2 <= y <= 1 + 0.2 cos(pi x), P2, 513 x 513
  nodes, dt = 1e-3, 400 steps, d_u = 0.05, checkpoints every 50 steps): adjoint
  gradients through torch.autograd against central finite differences of the
  GPU forward map, to 1e-5, for U_0 and d_u, and for f (along a smooth direction)
  and r at the workload's f = 0, r = 0.

Tolerances: every solve stops at an FP64 relative residual of 1e-11 (1e-12 on
the small grids); the gradients inherit that accuracy times the conditioning of
S = M + d_u tau A, which is mass-dominated (cond ~ 1 + d_u tau lam_max ~ 1e2).
"""
import numpy as np
import pytest

from oracle.heat import HeatOperators, imex_forward, imex_adjoint, loss, imex_forward_src, imex_adjoint_src
from paper_2109_01173_gb300.inputs import Profile, smoothed_uniform, heat_config

pytestmark = pytest.mark.gpu

G1 = Profile(c2=0.1)
G2 = Profile(c0=1.0, ca=0.2, cf=1.0)


@pytest.fixture(scope="module")
def mods():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    torch.cuda.set_device(0)
    import paper_2109_01173_gb300.mofem as mf
    import paper_2109_01173_gb300.adjoint as adj
    return torch, mf, adj


@pytest.mark.parametrize("k,n,bc,prec", [(2, 17, "neumann", "fp16"), (2, 17, "dirichlet", "fp64"),
                                         (0, 20, "neumann", "bf16"), (1, 13, "dirichlet", "tf32")])
def test_heat_forward_and_adjoint_vs_oracle(mods, k, n, bc, prec):
    torch, mf, adj = mods
    d, tau, steps, every = 0.05, 1e-3, 12, 5
    ops = HeatOperators(G1, G2, k, n, bc)
    q = ops.q
    U0 = smoothed_uniform(q, 1)
    T = smoothed_uniform(q, 2)
    states = imex_forward(ops, d, tau, U0, steps)
    J, dJ = loss(states[-1], T)
    gU_o, gd_o = imex_adjoint(ops, d, tau, states, dJ)

    setup = adj.HeatSetup(G1, G2, k, n, tau, bc=mf.NEUMANN if bc == "neumann" else mf.DIRICHLET,
                          precision=prec, rtol=1e-12)
    U0t = torch.tensor(U0[None], device="cuda", requires_grad=True)
    dut = torch.tensor(d, dtype=torch.float64, device="cuda", requires_grad=True)
    UN = adj.heat_imex(U0t, dut, setup, steps, every)
    assert np.abs(UN[0].detach().cpu().numpy() - states[-1]).max() <= 1e-9 * np.abs(states[-1]).max()
    Tt = torch.tensor(T[None], device="cuda")
    Jt = ((UN - Tt) ** 2).sum()
    Jt.backward()
    gU = U0t.grad[0].cpu().numpy()
    assert abs(Jt.item() - J) <= 1e-9 * J
    assert np.linalg.norm(gU - gU_o) <= 1e-7 * np.linalg.norm(gU_o)
    assert abs(dut.grad.item() - gd_o) <= 1e-7 * abs(gd_o)
    setup.close()


@pytest.mark.parametrize("k,n,bc,prec", [(2, 17, "neumann", "fp16"), (1, 13, "dirichlet", "fp64"),
                                         (0, 20, "dirichlet", "bf16")])
def test_heat_source_reaction_gradients_vs_oracle(mods, k, n, bc, prec):
    torch, mf, adj = mods
    d, tau, steps, every, r = 0.05, 1e-3, 12, 5, 0.8
    ops = HeatOperators(G1, G2, k, n, bc)
    q = ops.q
    U0, T = smoothed_uniform(q, 3), smoothed_uniform(q, 4)
    F = np.random.default_rng(n).standard_normal((n, n))
    states = imex_forward_src(ops, d, tau, U0, steps, F, r)
    J, dJ = loss(states[-1], T)
    gU_o, gd_o, gF_o, gr_o = imex_adjoint_src(ops, d, tau, r, states, dJ)

    setup = adj.HeatSetup(G1, G2, k, n, tau, bc=mf.NEUMANN if bc == "neumann" else mf.DIRICHLET,
                          precision=prec, rtol=1e-12)
    U0t = torch.tensor(U0[None], device="cuda", requires_grad=True)
    dut = torch.tensor(d, dtype=torch.float64, device="cuda", requires_grad=True)
    Ft = torch.tensor(F[None], device="cuda", requires_grad=True)
    rt = torch.tensor(r, dtype=torch.float64, device="cuda", requires_grad=True)
    UN = adj.heat_imex(U0t, dut, setup, steps, every, F=Ft, r=rt)
    assert np.abs(UN[0].detach().cpu().numpy() - states[-1]).max() <= 1e-9 * np.abs(states[-1]).max()
    Jt = ((UN - torch.tensor(T[None], device="cuda")) ** 2).sum()
    Jt.backward()
    assert abs(Jt.item() - J) <= 1e-9 * J
    assert np.linalg.norm(U0t.grad[0].cpu().numpy() - gU_o) <= 1e-7 * np.linalg.norm(gU_o)
    assert np.linalg.norm(Ft.grad[0].cpu().numpy() - gF_o) <= 1e-7 * np.linalg.norm(gF_o)
    assert abs(dut.grad.item() - gd_o) <= 1e-7 * abs(gd_o)
    assert abs(rt.grad.item() - gr_o) <= 1e-7 * abs(gr_o)
    setup.close()


def test_heat_adjoint_vs_finite_differences_workload(mods):
    """The differentiation workload at full size: adjoint vs central differences to 1e-5."""
    torch, mf, adj = mods
    cfg = heat_config()
    setup = adj.HeatSetup(cfg["g1"], cfg["g2"], cfg["k"], cfg["n"], cfg["tau"], bc=mf.NEUMANN, precision="fp16",
                          rtol=1e-11)
    q = cfg["n"]
    steps, every, d = cfg["steps"], cfg["every"], cfg["d_u"]
    U0 = torch.tensor(smoothed_uniform(q, 0)[None], device="cuda")
    with torch.no_grad():   # target: a seeded run from another initial field
        T = adj.heat_imex(torch.tensor(smoothed_uniform(q, 1)[None], device="cuda"),
                          torch.tensor(d, dtype=torch.float64), setup, steps, every)

    def J(U, dd):
        with torch.no_grad():
            UN = adj.heat_imex(U, torch.tensor(dd, dtype=torch.float64), setup, steps, every)
            return float(((UN - T) ** 2).sum().item())

    U0g = U0.clone().requires_grad_(True)
    dut = torch.tensor(d, dtype=torch.float64, device="cuda", requires_grad=True)
    UN = adj.heat_imex(U0g, dut, setup, steps, every)
    Jt = ((UN - T) ** 2).sum()
    Jt.backward()
    # d_u: relative step 1e-4 (truncation ~1e-8 relative)
    eps = 1e-4 * d
    fd = (J(U0, d + eps) - J(U0, d - eps)) / (2 * eps)
    assert abs(dut.grad.item() - fd) <= 1e-5 * abs(fd), (dut.grad.item(), fd)
    # U_0 along a smooth seeded direction (J is quadratic in U_0)
    V = torch.tensor(smoothed_uniform(q, 7)[None] - 0.5, device="cuda")
    V = V / V.norm()
    e = 1e-2
    fdv = (J(U0 + e * V, d) - J(U0 - e * V, d)) / (2 * e)
    adv = float((U0g.grad * V).sum().item())
    assert abs(adv - fdv) <= 1e-5 * abs(fdv), (adv, fdv)
    setup.close()


def test_heat_source_reaction_adjoint_vs_finite_differences_workload(mods):
    """The differentiation workload at f = 0, r = 0 with f and r as differentiable inputs:
    dJ/df along a smooth seeded direction against central differences (J is quadratic in
    f), and dJ/dr against its closed form, both to 1e-5.  With f = 0 every step multiplies
    the state by (1 - tau r) S^-1 M~, so U_N(r) = (1 - tau r)^N U_N(0) and
    dJ/dr(0) = -2 N tau <U_N(0) - T, U_N(0)> (central differences in r would carry a
    truncation error: J(r) is a polynomial of degree 2N in r with large higher
    derivatives on this workload)."""
    torch, mf, adj = mods
    cfg = heat_config()
    setup = adj.HeatSetup(cfg["g1"], cfg["g2"], cfg["k"], cfg["n"], cfg["tau"], bc=mf.NEUMANN, precision="fp16",
                          rtol=1e-11)
    n = q = cfg["n"]
    steps, every, d = cfg["steps"], cfg["every"], cfg["d_u"]
    dut = torch.tensor(d, dtype=torch.float64, device="cuda")
    U0 = torch.tensor(smoothed_uniform(q, 0)[None], device="cuda")
    with torch.no_grad():
        T = adj.heat_imex(torch.tensor(smoothed_uniform(q, 1)[None], device="cuda"), dut, setup, steps, every)
    F0 = torch.zeros((1, n, n), dtype=torch.float64, device="cuda")

    def J(F, r):
        with torch.no_grad():
            UN = adj.heat_imex(U0, dut, setup, steps, every, F=F, r=torch.tensor(r, dtype=torch.float64))
            return float(((UN - T) ** 2).sum().item())

    Fg = F0.clone().requires_grad_(True)
    rg = torch.tensor(0.0, dtype=torch.float64, device="cuda", requires_grad=True)
    UN = adj.heat_imex(U0, dut, setup, steps, every, F=Fg, r=rg)
    ((UN - T) ** 2).sum().backward()
    W = torch.tensor(smoothed_uniform(n, 9)[None] - 0.5, device="cuda")
    W = W / W.norm()
    e = 1e-2   # J is quadratic in f
    fdw = (J(F0 + e * W, 0.0) - J(F0 - e * W, 0.0)) / (2 * e)
    adw = float((Fg.grad * W).sum().item())
    assert abs(adw - fdw) <= 1e-5 * abs(fdw), (adw, fdw)
    with torch.no_grad():
        UN0 = adj.heat_imex(U0, dut, setup, steps, every)
    closed = -2.0 * steps * cfg["tau"] * float(((UN0 - T) * UN0).sum().item())
    assert abs(rg.grad.item() - closed) <= 1e-5 * abs(closed), (rg.grad.item(), closed)
    setup.close()
