"""GPU parity of libmofem (through the C ABI) against the FP64 CPU oracle.

Covers every hot-path step: operator apply (FP64 and FP32), right-hand side,
reduced-approach preconditioner (FP64 DGEMM form and tcgen05 TF32/BF16 form),
MO-PCG solves (FP64 form and mixed form with refinement), batching, the IMEX
step, error reporting, determinism, and the full-size P2 2049 x 2049 workload
of bench.py (sampled outputs and size-independent properties).

Tolerances (written per test) follow from the arithmetic:
* FP64 apply / rhs: a sum of at most 8 * 81 products -> 1e-13 of max |Y|.
* FP32 apply: forward error of the two-stage sums in difference form
  (row sum x_r + sum A_rj (x_j - x_r)), elementwise
  |err| <= 2 (P + NT P + 2) u32 (|S| |X| |T|^T)  with u32 = 2^-24.
* tensor-core preconditioner vs FP64: operands rounded to BF16 (u = 2^-9),
  truncated to TF32 (2^-10) or rounded to FP16 (2^-11, residual operand scaled
  to unit RMS) in four chained GEMMs: Frobenius 2.5e-2 / 1.5e-2 / 1.5e-2.
* solves: relative error <= 1e-8 against the oracle's 1e-13-residual solution
  and FP64 true residual <= rtol = 1e-10.
"""
import numpy as np
import pytest

from oracle.operator import Problem, apply_terms, rhs, apply_entry
from oracle import pcg
from paper_2109_01173_gb300.inputs import Profile, ZERO, SIN_TOP, fourier_f, metric_instance
from ddref import residual_dd

pytestmark = pytest.mark.gpu

TWO = (Profile(c2=0.1), Profile(c0=1.0, ca=0.2, cf=1.0))
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def mf():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    torch.cuda.set_device(0)
    import paper_2109_01173_gb300.mofem as m
    return m


def torch_():
    import torch
    return torch


def live(P):
    return [(S, T) for S, T in P.terms() if abs(S).sum() > 0]


def dom(name):
    return (ZERO, SIN_TOP) if name == "one" else TWO


# (k, n, domain, bc): several 128-column tiles and ~65-row tiles with ragged tails
APPLY_CASES = [(2, 301, "one", 0), (1, 200, "two", 1), (4, 161, "two", 0), (0, 150, "one", 0),
               (3, 151, "one", 1), (2, 263, "two", 1), (1, 5, "one", 0), (2, 5, "two", 0)]


@pytest.mark.parametrize("k,n,dname,bc", APPLY_CASES)
def test_apply_parity(mf, k, n, dname, bc):
    torch = torch_()
    g1, g2 = dom(dname)
    P = Problem(g1, g2, k, n, 0.7, bc="dirichlet" if bc == 0 else "neumann")
    h = mf.Handle(g1, g2, k, n, 0.7, bc=bc)
    q = h.q
    X = np.random.default_rng(k * 1000 + n).standard_normal((q, q))
    Yo = apply_terms(live(P), X)
    # FP64 (padded leading dimension exercises ld != q)
    ld = q + 3
    Xt = torch.zeros((q, ld), dtype=torch.float64, device="cuda")
    Xt[:, :q] = torch.tensor(X, device="cuda")
    Yt = torch.full((q, ld), 7.0, dtype=torch.float64, device="cuda")
    h.apply(Xt, Yt, "fp64", ld=ld)
    Y = Yt[:, :q].cpu().numpy()
    assert np.abs(Y - Yo).max() <= 1e-13 * np.abs(Yo).max()
    assert torch.all(Yt[:, q:] == 7.0)                       # padding untouched
    # FP32: elementwise forward-error bound of the two-stage sums
    X32 = X.astype(np.float32)
    Yo32 = apply_terms(live(P), X32.astype(np.float64))
    absb = apply_terms([(abs(S), abs(T)) for S, T in live(P)], np.abs(X32.astype(np.float64)))
    Pw = 2 * max(k, 1) + 1
    bound = 2 * (Pw + h.n_terms * Pw + 2) * U32 * absb
    Xf = torch.tensor(X32, device="cuda")
    Yf = torch.zeros_like(Xf)
    h.apply(Xf, Yf, "bf16")
    err = np.abs(Yf.cpu().numpy().astype(np.float64) - Yo32)
    assert np.all(err <= bound + 1e-30)
    h.close()


@pytest.mark.parametrize("k,n,dname,bc", APPLY_CASES[:5])
def test_rhs_parity(mf, k, n, dname, bc):
    torch = torch_()
    g1, g2 = dom(dname)
    P = Problem(g1, g2, k, n, 0.7, bc="dirichlet" if bc == 0 else "neumann")
    h = mf.Handle(g1, g2, k, n, 0.7, bc=bc)
    F = np.random.default_rng(n).standard_normal((n, n))
    Bt = torch.zeros((h.q, h.q), dtype=torch.float64, device="cuda")
    h.rhs(torch.tensor(F, device="cuda"), Bt)
    Bo = rhs(P, F)
    assert np.abs(Bt.cpu().numpy() - Bo).max() <= 1e-13 * np.abs(Bo).max()
    h.close()


@pytest.mark.parametrize("k,n,dname,bc", [(2, 301, "one", 0), (1, 200, "two", 1), (4, 161, "two", 0),
                                          (0, 150, "one", 0), (2, 5, "one", 0)])
def test_precond_parity(mf, k, n, dname, bc):
    torch = torch_()
    g1, g2 = dom(dname)
    P = Problem(g1, g2, k, n, 0.7, bc="dirichlet" if bc == 0 else "neumann")
    h = mf.Handle(g1, g2, k, n, 0.7, bc=bc)
    E1, E2, F1, F2 = P.pencils()
    Zo = pcg.ReducedSylvester(E1, E2, F1, F2)(np.random.default_rng(1).standard_normal((h.q, h.q)))
    R = np.random.default_rng(1).standard_normal((h.q, h.q))
    Zt = torch.zeros((h.q, h.q), dtype=torch.float64, device="cuda")
    h.precond(torch.tensor(R, device="cuda"), Zt, "fp64")
    Z = Zt.cpu().numpy()
    assert np.linalg.norm(Z - Zo) <= 1e-9 * np.linalg.norm(Zo)
    back = E1 @ Z @ F1.T + E2 @ Z @ F2.T
    assert np.linalg.norm(back - R) <= 1e-9 * np.linalg.norm(R)
    for prec, tol in (("bf16", 2.5e-2), ("tf32", 1.5e-2), ("fp16", 1.5e-2)):
        Zf = torch.zeros((h.q, h.q), dtype=torch.float32, device="cuda")
        h.precond(torch.tensor(R, dtype=torch.float32, device="cuda"), Zf, prec)
        Zm = Zf.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(Zm - Zo) <= tol * np.linalg.norm(Zo), prec
    h.close()


# ---- one search-direction step: Q = Z + beta Q_prev, LQ = L(Q), alpha = rz / <Q, LQ> ----------
# FP32 cases run the packed-FP32 kernel (K = 1..3 with 5 terms, K = 1, 2 with 8 terms) or the
# scalar one (larger bands); FP64 runs the FP64 kernel.  Several 128-column and 40-row tiles
# with ragged tails, ld > q (padding must come back zero), two instances per handle.
DIRECTION_CASES = [(2, 301, "one", 0), (2, 263, "two", 1), (1, 200, "two", 1), (0, 150, "one", 0),
                   (3, 151, "one", 1), (4, 161, "two", 0), (2, 5, "one", 0), (1, 7, "two", 1)]


def _direction_case(mf, k, n, dname, bc, prec, ld_extra):
    torch = torch_()
    g1, g2 = dom(dname)
    gam = [0.7, 2.5]
    h = mf.Handle([g1, g1], [g2, g2], k, n, gam, bc=bc)
    q = h.q
    dt = torch.float64 if prec == "fp64" else torch.float32
    npdt = np.float64 if prec == "fp64" else np.float32
    ld = ((q + 3) // 4) * 4 + ld_extra
    rng = np.random.default_rng(7 * n + k)
    Z = rng.standard_normal((2, q, q)).astype(npdt)
    Qp = rng.standard_normal((2, q, q)).astype(npdt)
    beta, rz = [0.37, -1.25], [2.0, 0.5]

    def dev(A):
        t = torch.zeros((2, q, ld), dtype=dt, device="cuda")
        t[:, :, :q] = torch.tensor(A, device="cuda")
        return t
    Zt, Qpt = dev(Z), dev(Qp)
    Qt = torch.full((2, q, ld), 7.0, dtype=dt, device="cuda")
    LQt = torch.full((2, q, ld), 7.0, dtype=dt, device="cuda")
    alpha, code = h.pcg_direction(Zt, Qpt, beta, rz, Qt, LQt, precision=prec, ld=ld)
    assert code == 0
    Qg = Qt[:, :, :q].cpu().numpy().astype(np.float64)
    LQg = LQt[:, :, :q].cpu().numpy().astype(np.float64)
    u = 2.0 ** -53 if prec == "fp64" else U32
    Pw = 2 * max(k, 1) + 1
    for i in range(2):
        P = Problem(g1, g2, k, n, gam[i], bc="dirichlet" if bc == 0 else "neumann")
        b = float(npdt(beta[i]))
        Qe = Z[i].astype(np.float64) + b * Qp[i].astype(np.float64)
        # one rounding on the GPU (two in the FP64 reference): relative to the operands
        mag = np.abs(Z[i].astype(np.float64)) + np.abs(b * Qp[i].astype(np.float64))
        assert np.all(np.abs(Qg[i] - Qe) <= 2 * u * mag + 1e-300), i
        Yo = apply_terms(live(P), Qg[i])
        absb = apply_terms([(abs(S), abs(T)) for S, T in live(P)], np.abs(Qg[i]))
        bound = 2 * (Pw + h.n_terms * Pw + 2) * u * absb
        assert np.all(np.abs(LQg[i] - Yo) <= bound + 1e-300), i
        qlq = float(np.sum(Qg[i] * LQg[i]))
        tol = 64 * u * float(np.sum(np.abs(Qg[i] * LQg[i])))
        assert abs(rz[i] / alpha[i] - qlq) <= tol, (i, rz[i] / alpha[i], qlq)
    # padding columns: zero where the kernel's tiles reach, untouched beyond
    for T in (Qt, LQt):
        pad = T[:, :, q:].cpu().numpy()
        reach = min(ld, ((q + 127) // 128) * 128) - q
        assert np.all((pad[:, :, :reach] == 0) | (pad[:, :, :reach] == 7.0))
        assert np.all(pad[:, :, reach:] == 7.0)
    h.close()


@pytest.mark.parametrize("k,n,dname,bc", DIRECTION_CASES)
@pytest.mark.parametrize("prec", ["fp16", "fp64"])
def test_pcg_direction_parity(mf, k, n, dname, bc, prec):
    _direction_case(mf, k, n, dname, bc, prec, ld_extra=0)


def test_pcg_direction_wide_ld(mf):
    _direction_case(mf, 2, 301, "one", 0, "tf32", ld_extra=200)


def test_pcg_direction_breakdown(mf):
    """<Q, L(Q)> = 0 (zero direction): BREAKDOWN, alpha = 0, nothing non-finite."""
    torch = torch_()
    h = mf.Handle([ZERO, ZERO], [SIN_TOP, SIN_TOP], 2, 65, [1.0, 1.0])
    q = h.q
    ld = ((q + 3) // 4) * 4
    Zt = torch.zeros((2, q, ld), dtype=torch.float32, device="cuda")
    Zt[1, 3, 5] = 1.0
    Qp = torch.zeros_like(Zt)
    Qt, LQt = torch.zeros_like(Zt), torch.zeros_like(Zt)
    alpha, code = h.pcg_direction(Zt, Qp, [0.0, 0.0], [1.0, 1.0], Qt, LQt, precision="bf16", ld=ld, check=False)
    assert code == mf.ERR_BREAKDOWN
    assert alpha[0] == 0.0 and alpha[1] > 0.0
    assert torch.isfinite(LQt).all()
    h.close()


SOLVE_CASES = [(2, 129, "one", 0, 1.0), (1, 97, "two", 1, 2.0), (4, 81, "two", 0, 0.0), (0, 101, "one", 0, 1.0),
               (3, 64, "one", 1, 0.5)]


@pytest.mark.parametrize("k,n,dname,bc,gamma", SOLVE_CASES)
@pytest.mark.parametrize("prec", ["fp64", "bf16", "tf32", "fp16"])
def test_solve_parity(mf, k, n, dname, bc, gamma, prec):
    torch = torch_()
    g1, g2 = dom(dname)
    P = Problem(g1, g2, k, n, gamma, bc="dirichlet" if bc == 0 else "neumann")
    F = fourier_f(g1, g2, n, seed=n + k)
    Uo, _ = pcg.solve(P, F, rtol=1e-13)
    h = mf.Handle(g1, g2, k, n, gamma, bc=bc)
    U = torch.zeros((h.q, h.q), dtype=torch.float64, device="cuda")
    info, code = h.pcg_solve(torch.tensor(F, device="cuda"), U, rtol=1e-10, max_iter=400, precision=prec)
    assert code == 0 and info.rel_residual <= 1e-10
    Ug = U.cpu().numpy()
    assert np.linalg.norm(Ug - Uo) <= 1e-8 * np.linalg.norm(Uo)
    # the oracle's own FP64 residual of the GPU solution
    B = rhs(P, F)
    assert np.linalg.norm(B - apply_terms(live(P), Ug)) <= 1.5e-10 * np.linalg.norm(B)
    h.close()


def test_batched_solve(mf):
    torch = torch_()
    n, k = 97, 2
    g2s = [Profile(c0=1.0, sa=0.1, sf=1), Profile(c0=1.0, sa=0.25, sf=2), Profile(c0=1.0, sa=0.3, sf=3)]
    gam = [0.0, 3.5, 9.0]
    Fs = [fourier_f(ZERO, g, n, seed=i) for i, g in enumerate(g2s)]
    h = mf.Handle([ZERO] * 3, g2s, k, n, gam)
    U = torch.zeros((3, h.q, h.q), dtype=torch.float64, device="cuda")
    info, code = h.pcg_solve(torch.tensor(np.stack(Fs), device="cuda"), U, rtol=1e-10, max_iter=400,
                             precision="bf16")
    assert code == 0
    for i in range(3):
        Uo, _ = pcg.solve(Problem(ZERO, g2s[i], k, n, gam[i]), Fs[i], rtol=1e-13)
        assert np.linalg.norm(U[i].cpu().numpy() - Uo) <= 1e-8 * np.linalg.norm(Uo), i
    h.close()


def test_uniform_batch_sixteen_instances(mf):
    """The uniform-batch form at 16 instances (gamma ~ U[0,10], top 1 + a sin(2 pi b x), each
    with its own seeded Fourier f; the generator of the bench's batch sweep) at P2, 65 x 65
    nodes: every instance of one mixed FP16 solve against its own FP64 oracle solve."""
    from paper_2109_01173_gb300.inputs import batch_instances
    torch = torch_()
    ins = batch_instances(16, n=65, k=2, seed0=1000)
    h = mf.Handle([i["g1"] for i in ins], [i["g2"] for i in ins], 2, 65, [i["gamma"] for i in ins])
    U = torch.zeros((16, h.q, h.q), dtype=torch.float64, device="cuda")
    F = torch.tensor(np.stack([i["F"] for i in ins]), dtype=torch.float64, device="cuda")
    info, code = h.pcg_solve(F, U, rtol=1e-10, max_iter=400, precision="fp16")
    assert code == 0 and info.rel_residual <= 1e-10
    for i, I in enumerate(ins):
        Uo, _ = pcg.solve(Problem(I["g1"], I["g2"], 2, 65, I["gamma"]), I["F"], rtol=1e-13)
        assert np.linalg.norm(U[i].cpu().numpy() - Uo) <= 1e-8 * np.linalg.norm(Uo), i
    h.close()


@pytest.mark.parametrize("prec", ["fp16", "fp64"])
def test_zero_right_hand_side(mf, prec):
    """F = 0 gives U = 0 at once (the initialisation marks the instance inactive), alone
    and as one instance of a batch whose other instances solve as they do alone."""
    torch = torch_()
    n, k = 97, 2
    h1 = mf.Handle(ZERO, SIN_TOP, k, n, 1.0)
    U1 = torch.full((h1.q, h1.q), 0.0, dtype=torch.float64, device="cuda")
    info, code = h1.pcg_solve(torch.zeros((n, n), dtype=torch.float64, device="cuda"), U1, rtol=1e-10,
                              max_iter=100, precision=prec, check=False)
    assert code == mf.OK and info.iterations == 0 and info.rel_residual == 0.0
    assert bool((U1 == 0).all())
    h1.close()
    g2s = [Profile(c0=1.0, sa=0.1, sf=1), Profile(c0=1.0, sa=0.25, sf=2), Profile(c0=1.0, sa=0.2, sf=1),
           Profile(c0=1.0, sa=0.3, sf=3)]
    gam = [1.0, 3.5, 2.0, 9.0]
    Fs = [fourier_f(ZERO, g, n, seed=i) for i, g in enumerate(g2s)]
    Fs[2] = np.zeros((n, n))
    h = mf.Handle([ZERO] * 4, g2s, k, n, gam)
    U = torch.zeros((4, h.q, h.q), dtype=torch.float64, device="cuda")
    info, code = h.pcg_solve(torch.tensor(np.stack(Fs), device="cuda"), U, rtol=1e-10, max_iter=400,
                             precision=prec)
    assert code == mf.OK and info.rel_residual <= 1e-10
    assert bool((U[2] == 0).all())
    for i in (0, 1, 3):
        Uo, _ = pcg.solve(Problem(ZERO, g2s[i], k, n, gam[i]), Fs[i], rtol=1e-13)
        assert np.linalg.norm(U[i].cpu().numpy() - Uo) <= 1e-8 * np.linalg.norm(Uo), i
    h.close()


def test_deterministic(mf):
    torch = torch_()
    inst = metric_instance(n=129, k=2, seed=3)
    h = mf.Handle(inst["g1"], inst["g2"], 2, 129, 1.0)
    F = torch.tensor(inst["F"], device="cuda")
    out = []
    for _ in range(2):
        U = torch.zeros((h.q, h.q), dtype=torch.float64, device="cuda")
        h.pcg_solve(F, U, rtol=1e-10, max_iter=300, precision="bf16")
        out.append(U.cpu().numpy())
    assert np.array_equal(out[0], out[1])
    h.close()


def test_error_reporting(mf):
    torch = torch_()
    inst = metric_instance(n=65, k=1, seed=0)
    h = mf.Handle(inst["g1"], inst["g2"], 1, 65, 1.0, opts=mf.make_opts(max_outer=1))
    F = torch.tensor(inst["F"], device="cuda")
    U = torch.zeros((h.q, h.q), dtype=torch.float64, device="cuda")
    info, code = h.pcg_solve(F, U, rtol=1e-10, max_iter=1, precision="bf16", check=False)
    assert code == mf.ERR_NOT_CONVERGED and info.iterations == 1
    Fn = F.clone()
    Fn[10, 10] = float("nan")
    U.zero_()
    info, code = h.pcg_solve(Fn, U, rtol=1e-10, max_iter=50, precision="fp64", check=False)
    assert code == mf.ERR_NONFINITE
    h.close()


@pytest.mark.parametrize("bc", [0, 1])
def test_imex_step(mf, bc):
    """One IMEX Euler step (Sec. 6): (M + d tau A) U1 = M (U0 + tau f), stop ||R_s|| <= tau ||R_0||."""
    torch = torch_()
    n, k, du, tau = 65, 2, 0.05, 1e-3
    g1, g2 = Profile(c2=0.1), Profile(c0=1.0, ca=0.2, cf=1.0)
    gam = 1.0 / (du * tau)
    P = Problem(g1, g2, k, n, gam, bc="dirichlet" if bc == 0 else "neumann")
    q = P.q
    rng = np.random.default_rng(0)
    U0 = rng.uniform(0, 1, (q, q))
    Fn = rng.standard_normal((n, n))
    h = mf.Handle(g1, g2, k, n, gam, bc=bc)
    Ut = torch.zeros((q, q), dtype=torch.float64, device="cuda")
    info, code = h.imex_step(du, tau, torch.tensor(U0, device="cuda"), torch.tensor(Fn, device="cuda"), Ut,
                             precision="bf16")
    assert code == 0
    off = 1 if bc == 0 else 0
    Fbar = gam * tau * Fn
    Fbar[off:off + q, off:off + q] += gam * U0
    B = rhs(P, Fbar)
    L = lambda X: apply_terms(live(P), X)
    r0 = np.linalg.norm(B - L(U0))
    r1 = np.linalg.norm(B - L(Ut.cpu().numpy()))
    assert r1 <= tau * r0
    h.close()


# ---- full-size workload of bench.py: P2, 2049 x 2049 nodes -----------------------------
@pytest.fixture(scope="module")
def full(mf):
    torch = torch_()
    inst = metric_instance(n=2049, k=2, seed=0)
    P = Problem(inst["g1"], inst["g2"], 2, 2049, 1.0)
    h = mf.Handle(inst["g1"], inst["g2"], 2, 2049, 1.0)
    yield inst, P, h
    h.close()


def test_full_size_sampled_apply(mf, full):
    torch = torch_()
    inst, P, h = full
    q = h.q
    X = np.random.default_rng(11).standard_normal((q, q))
    Xt = torch.tensor(X, device="cuda")
    Yt = torch.zeros_like(Xt)
    h.apply(Xt, Yt, "fp64")
    Y = Yt.cpu().numpy()
    terms = live(P)
    rng = np.random.default_rng(12)
    pts = [(0, 0), (q - 1, q - 1), (0, q - 1), (q - 1, 0), (127, 128), (64, 2046)]
    pts += [tuple(p) for p in rng.integers(0, q, size=(40, 2))]
    scale = np.abs(Y).max()
    for a, b in pts:
        assert abs(Y[a, b] - apply_entry(terms, X, a, b)) <= 1e-13 * scale, (a, b)


def test_full_size_solve(mf, full):
    torch = torch_()
    inst, P, h = full
    F = torch.tensor(inst["F"], device="cuda")
    U = torch.zeros((h.q, h.q), dtype=torch.float64, device="cuda")
    info, code = h.pcg_solve(F, U, rtol=1e-10, max_iter=500, precision="bf16")
    assert code == 0
    Ug = U.cpu().numpy()
    B = rhs(P, inst["F"])
    res = np.linalg.norm(B - apply_terms(live(P), Ug)) / np.linalg.norm(B)
    assert res <= 1.5e-10
    U64 = torch.zeros_like(U)
    info64, code64 = h.pcg_solve(F, U64, rtol=1e-10, max_iter=500, precision="fp64")
    assert code64 == 0
    assert float(((U64 - U).norm() / U64.norm()).item()) <= 1e-8


def _true_rel(h, F, U):
    """||B - L(U)|| / ||B|| per instance with the library's FP64 (difference-form) apply."""
    torch = torch_()
    B = torch.zeros_like(U)
    h.rhs(F, B)
    Y = torch.zeros_like(U)
    h.apply(U, Y, "fp64")
    R = (B - Y).reshape(U.shape[0] if U.dim() == 3 else 1, -1)
    return (R.norm(dim=1) / B.reshape(R.shape).norm(dim=1)).tolist()


def _solve_both(mf, g1, g2, k, n, gam, bc, F, prec, rtol=1e-10):
    """The same solve with the residual updated in double-float arithmetic after every
    step (default) and recomputed in FP64 after every step (FLAG_TRUE_RESIDUAL)."""
    torch = torch_()
    B = len(g1)
    out = []
    for flags in (0, mf.FLAG_TRUE_RESIDUAL):
        h = mf.Handle(g1, g2, k, n, gam, bc=bc, opts=mf.make_opts(flags=flags))
        U = torch.zeros((B, h.q, h.q), dtype=torch.float64, device="cuda")
        info, code = h.pcg_solve(F, U, rtol=rtol, max_iter=500, precision=prec)
        assert code == 0 and info.outer_steps >= 2
        out.append((U, info.rel_residual, _true_rel(h, F, U)))
        h.close()
    return out


def test_residual_update_full_size(mf):
    """Bench workload (P2, 2049 x 2049 nodes, 4 instances, rtol 1e-10).  The two runs
    agree to 1e-8 (their first steps' residuals differ by the FP64 evaluation noise, so
    the later inner solves start from slightly different right-hand sides); each reported
    residual differs from an FP64 recomputation only by that recomputation's evaluation
    noise (u q^2 / pi^2 = 4.7e-11 of ||B|| at q = 2047, the t-pass mass product rounded to
    FP64 and then second-differenced); the target holds on the recomputed residual."""
    torch = torch_()
    insts = [metric_instance(n=2049, k=2, seed=s) for s in range(4)]
    F = torch.tensor(np.stack([i["F"] for i in insts]), device="cuda")
    (U0, rep0, rel0), (U1, rep1, rel1) = _solve_both(mf, [i["g1"] for i in insts], [i["g2"] for i in insts], 2,
                                                     2049, [1.0] * 4, 0, F, "fp16")
    assert float(((U0 - U1).norm() / U1.norm()).item()) <= 1e-8
    assert max(rel0) <= 1e-10
    assert abs(max(rel1) - rep1) <= 1e-13, (rep1, rel1)
    noise = 2.0 ** -53 * 2047 ** 2 / np.pi ** 2
    assert abs(max(rel0) - rep0) <= 2 * noise, (rep0, rel0)


@pytest.mark.parametrize("k,n,dname,bc,gamma", [(2, 257, "one", 0, 1.0), (1, 301, "two", 1, 2.0),
                                                 (3, 193, "two", 0, 0.5), (0, 257, "one", 1, 1.0)])
def test_residual_update_tracks_recomputed(mf, k, n, dname, bc, gamma):
    """Where the FP64 evaluation noise is small (u q^2 / pi^2 < 1e-12), the updated
    residual equals the recomputed one to 2e-12 of ||B||: an error of 1e-6 in the
    double-float L(d) (or a missed rounding of the iterate) would show at 1e-11."""
    torch = torch_()
    g1, g2 = dom(dname)
    F = torch.tensor(fourier_f(g1, g2, n, seed=n), device="cuda").unsqueeze(0)
    (U0, rep0, rel0), (U1, rep1, rel1) = _solve_both(mf, [g1], [g2], k, n, [gamma], bc, F, "bf16")
    assert float(((U0 - U1).norm() / U1.norm()).item()) <= 1e-8
    assert abs(rel0[0] - rep0) <= 2e-12, (rep0, rel0)
    assert abs(rel1[0] - rep1) <= 1e-13, (rep1, rel1)


@pytest.mark.parametrize("k,n", [(2, 2049), (1, 1025)])
def test_first_step_residual_double_float(mf, k, n):
    """One refinement step from zero: the residual B - L(U) that the solver carries
    (double-float difference form with exact row sums and input differences) against
    the same residual of the same iterate in double-double arithmetic on the library's
    own FP64 coefficients.  The step cancels R to ~1e-5 of B; the carried norm agrees to
    5e-12 of ||B|| (evaluation error ~2^-48 q), below the FP64 evaluation's own noise
    (u q^2 / pi^2, 4.7e-11 at q = 2047), which the recomputed residual shows."""
    torch = torch_()
    inst = metric_instance(n=n, k=k, seed=1)
    h = mf.Handle(inst["g1"], inst["g2"], k, n, 1.0, opts=mf.make_opts(max_outer=1))
    q = h.q
    F = torch.tensor(inst["F"], device="cuda")
    U = torch.zeros((q, q), dtype=torch.float64, device="cuda")
    info, code = h.pcg_solve(F, U, rtol=1e-10, max_iter=500, precision="fp16", check=False)
    assert info.outer_steps == 1 and 1e-7 < info.rel_residual < 1e-3
    Bt = torch.zeros_like(U)
    h.rhs(F, Bt)
    B = Bt.cpu().numpy()
    tb = mf.host_tables(inst["g1"], inst["g2"], k, n, 1.0)
    R = residual_dd(tb["S"], tb["T"], tb["K"], B, U.cpu().numpy())
    bn = np.linalg.norm(B)
    ref = np.linalg.norm(R) / bn
    assert abs(info.rel_residual - ref) <= 5e-12, (info.rel_residual, ref)
    rel64 = _true_rel(h, F.unsqueeze(0), U.unsqueeze(0))[0]   # FP64 GPU recomputation
    assert abs(rel64 - ref) <= 2 * 2.0 ** -53 * q * q / np.pi ** 2, (rel64, ref)
    h.close()


def test_residual_update_nonzero_guess(mf):
    """From a nonzero initial guess every step updates the residual (the first
    residual is recomputed before the loop): result against the oracle."""
    torch = torch_()
    k, n = 2, 129
    P = Problem(ZERO, SIN_TOP, k, n, 1.0)
    F = fourier_f(ZERO, SIN_TOP, n, seed=5)
    Uo, _ = pcg.solve(P, F, rtol=1e-13)
    h = mf.Handle(ZERO, SIN_TOP, k, n, 1.0)
    U = torch.tensor(Uo + 1e-3 * np.random.default_rng(2).standard_normal(Uo.shape), device="cuda")
    Ft = torch.tensor(F, device="cuda")
    info, code = h.pcg_solve(Ft, U, rtol=1e-10, max_iter=400, precision="bf16")
    assert code == 0
    assert np.linalg.norm(U.cpu().numpy() - Uo) <= 1e-8 * np.linalg.norm(Uo)
    rel = _true_rel(h, Ft.unsqueeze(0), U.unsqueeze(0))
    assert rel[0] <= 1e-10 and abs(rel[0] - info.rel_residual) <= 2e-12
    h.close()


def test_full_size_direction_batched(mf):
    """The PCG-form apply in the launch configuration of bench.py (P2, 2049 x 2049 nodes,
    four instances, FP32): new direction and L(Q) at sampled entries against the oracle's
    entry-wise apply, alpha against the FP64 dot of the returned arrays."""
    torch = torch_()
    n, k, B = 2049, 2, 4
    insts = [metric_instance(n=n, k=k, seed=s) for s in range(B)]
    h = mf.Handle([I["g1"] for I in insts], [I["g2"] for I in insts], k, n, [1.0] * B)
    q = h.q
    ld = ((q + 63) // 64) * 64
    g = torch.Generator(device="cuda").manual_seed(5)
    Zt = torch.zeros((B, q, ld), dtype=torch.float32, device="cuda")
    Qp = torch.zeros_like(Zt)
    Zt[:, :, :q] = torch.randn((B, q, q), generator=g, device="cuda")
    Qp[:, :, :q] = torch.randn((B, q, q), generator=g, device="cuda")
    Qt, LQt = torch.empty_like(Zt), torch.empty_like(Zt)
    beta, rz = [0.5, -0.25, 1.5, 0.0], [1.0, 2.0, 3.0, 4.0]
    alpha, code = h.pcg_direction(Zt, Qp, beta, rz, Qt, LQt, precision="fp16", ld=ld)
    assert code == 0
    rng = np.random.default_rng(13)
    pts = [(0, 0), (q - 1, q - 1), (0, q - 1), (q - 1, 0), (39, 127), (40, 128), (1919, 1920), (2046, 1023)]
    pts += [tuple(p) for p in rng.integers(0, q, size=(24, 2))]
    for i in range(B):
        P = Problem(insts[i]["g1"], insts[i]["g2"], k, n, 1.0)
        terms = live(P)
        Qg = Qt[i, :, :q].double().cpu().numpy()
        Zi = Zt[i, :, :q].double().cpu().numpy()
        Qpi = Qp[i, :, :q].double().cpu().numpy()
        b = float(np.float32(beta[i]))
        Qe = Zi + b * Qpi
        assert np.all(np.abs(Qg - Qe) <= 2 * U32 * (np.abs(Zi) + np.abs(b * Qpi)) + 1e-300)
        LQg = LQt[i, :, :q].double().cpu().numpy()
        absterms = [(abs(S), abs(T)) for S, T in terms]
        for a_, b_ in pts:
            ref = apply_entry(terms, Qg, a_, b_)
            bnd = 2 * (5 + h.n_terms * 5 + 2) * U32 * apply_entry(absterms, np.abs(Qg), a_, b_)
            assert abs(LQg[a_, b_] - ref) <= bnd + 1e-300, (i, a_, b_)
        qlq = float(np.sum(Qg * LQg))
        assert abs(rz[i] / alpha[i] - qlq) <= 64 * U32 * float(np.sum(np.abs(Qg * LQg))), i
        assert torch.all(Qt[i, :, q:] == 0) and torch.all(LQt[i, :, q:] == 0)
    h.close()


# ---- the paper's single-term product preconditioner (Sec. 5, Eq. vector_preconditioner) ----------
@pytest.mark.parametrize("k,n,dname", [(2, 65, "one"), (1, 97, "two"), (0, 64, "one"), (4, 81, "two")])
def test_product_preconditioner_parity(mf, k, n, dname):
    """Z = K_s[h]^-1 R (K_t + K_t[t^2])^-T by the reduced approach (standard eigenpairs,
    divisor lambda mu) against the oracle's banded direct solves."""
    torch = torch_()
    g1, g2 = dom(dname)
    P = Problem(g1, g2, k, n, 0.7)
    h = mf.Handle(g1, g2, k, n, 0.7, opts=mf.make_opts(pencil=mf.PENCIL_PRODUCT))
    R = np.random.default_rng(4).standard_normal((h.q, h.q))
    Zo = pcg.ProductPreconditioner(*P.product_factors())(R)
    Zt = torch.zeros((h.q, h.q), dtype=torch.float64, device="cuda")
    h.precond(torch.tensor(R, device="cuda"), Zt, "fp64")
    assert np.linalg.norm(Zt.cpu().numpy() - Zo) <= 1e-9 * np.linalg.norm(Zo)
    for prec, tol in (("tf32", 2e-2), ("bf16", 3e-2), ("fp16", 2e-2)):   # fp16 runs as TF32 for this form
        Zf = torch.zeros((h.q, h.q), dtype=torch.float32, device="cuda")
        h.precond(torch.tensor(R, dtype=torch.float32, device="cuda"), Zf, prec)
        Zm = Zf.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(Zm - Zo) <= tol * np.linalg.norm(Zo), prec
    h.close()


@pytest.mark.parametrize("prec", ["fp64", "tf32", "fp16"])
def test_product_preconditioner_solve(mf, prec):
    """MO-PCG with the product preconditioner: the solution of the oracle and, in the FP64
    form, the oracle's iteration count (same recurrences and stopping rule; the GPU form may add a
    residual-replacement restart) within two."""
    torch = torch_()
    k, n = 2, 65
    P = Problem(ZERO, SIN_TOP, k, n, 1.0)
    F = fourier_f(ZERO, SIN_TOP, n, 0)
    Uo, info_o = pcg.solve(P, F, precond='product', rtol=1e-13)
    _, info_10 = pcg.solve(P, F, precond='product', rtol=1e-10)
    h = mf.Handle(ZERO, SIN_TOP, k, n, 1.0, opts=mf.make_opts(pencil=mf.PENCIL_PRODUCT))
    U = torch.zeros((h.q, h.q), dtype=torch.float64, device="cuda")
    info, code = h.pcg_solve(torch.tensor(F, device="cuda"), U, rtol=1e-10, max_iter=2000, precision=prec)
    assert code == 0
    assert np.linalg.norm(U.cpu().numpy() - Uo) <= 1e-8 * np.linalg.norm(Uo)
    if prec == "fp64":
        assert abs(info.iterations - info_10["iterations"]) <= 2, (info.iterations, info_10["iterations"])
    h.close()
