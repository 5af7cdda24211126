"""GPU runs of the two elliptic test configurations besides the bench workload.

* Small configuration: plain MO-PCG on P1, 65 x 65 nodes, gamma = 1, Dirichlet,
  0 <= y <= 1 + 0.25 sin(2 pi x), f manufactured from u = sin(pi s) sin(pi t) plus
  seeded N(0, 1e-3) noise, rtol 1e-10: every precision against the oracle's 1e-13
  solution (relative error <= 1e-8), and the discrete solution against the
  manufactured u (P1 at h = 1/64: O(h^2) nodal error).
* Precision form at full size: P2 at n = 1025 and P4 at n = 2049, seeded 32-mode
  Fourier f.  The oracle cannot solve these in seconds, so: sampled operator
  outputs and every right-hand-side entry against the oracle, the mixed forms
  (BF16, TF32, FP16 GEMM operands) against the FP64 GPU form (relative difference
  <= 1e-8), and each solution's residual recomputed with the library's FP64 apply.
* The bench workload's batched right-hand side (P2 2049, 4 instances) against the
  oracle, every entry.
"""
import numpy as np
import pytest

from oracle.operator import Problem, apply_entry, rhs
from oracle import pcg
from paper_2109_01173_gb300.inputs import config_p1_65, metric_instance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mf():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    torch.cuda.set_device(0)
    import paper_2109_01173_gb300.mofem as m
    return m


def _true_rel(h, F, U):
    """||B - L(U)|| / ||B|| with the library's FP64 (difference-form) apply."""
    import torch
    B = torch.zeros_like(U)
    h.rhs(F, B)
    Y = torch.zeros_like(U)
    h.apply(U, Y, "fp64")
    return float((B - Y).norm() / B.norm())


def test_small_configuration(mf):
    import torch
    inst = config_p1_65(0)
    P = Problem(inst["g1"], inst["g2"], 1, 65, 1.0)
    Uo, _ = pcg.solve(P, inst["F"], rtol=1e-13)
    h = mf.Handle(inst["g1"], inst["g2"], 1, 65, 1.0)
    F = torch.tensor(inst["F"], device="cuda")
    for prec in ("fp64", "fp16", "bf16", "tf32"):
        U = torch.zeros((h.q, h.q), dtype=torch.float64, device="cuda")
        info, code = h.pcg_solve(F, U, rtol=1e-10, max_iter=500, precision=prec)
        assert code == 0 and info.rel_residual <= 1e-10, prec
        Ug = U.cpu().numpy()
        assert np.linalg.norm(Ug - Uo) <= 1e-8 * np.linalg.norm(Uo), prec
        assert _true_rel(h, F, U) <= 1e-10, prec
    # the discrete solution against the manufactured u at the interior nodes (the noise on
    # f is 1e-3 of its size; P1 nodal error at h = 1/64 is ~1e-3 of |u|)
    ue = inst["u_exact"][1:-1, 1:-1]
    err = np.linalg.norm(Uo - ue) / np.linalg.norm(ue)
    assert err <= 5e-3, err
    h.close()


@pytest.mark.parametrize("k,n", [(2, 1025), (4, 2049)])
def test_precision_form_full_size(mf, k, n):
    import torch
    inst = metric_instance(n=n, k=k, seed=0)
    h = mf.Handle(inst["g1"], inst["g2"], k, n, 1.0)
    q = h.q
    # sampled operator outputs against the oracle
    P = Problem(inst["g1"], inst["g2"], k, n, 1.0)
    terms = [(S, T) for S, T in P.terms() if abs(S).sum() > 0]
    X = np.random.default_rng(21).standard_normal((q, q))
    Xt = torch.tensor(X, device="cuda")
    Yt = torch.zeros_like(Xt)
    h.apply(Xt, Yt, "fp64")
    Y = Yt.cpu().numpy()
    rng = np.random.default_rng(22)
    pts = [(0, 0), (q - 1, q - 1), (0, q - 1), (q - 1, 0), (q // 2, q // 2 + 1)]
    pts += [tuple(p) for p in rng.integers(0, q, size=(30, 2))]
    scale = np.abs(Y).max()
    for a, b in pts:
        assert abs(Y[a, b] - apply_entry(terms, X, a, b)) <= 1e-13 * scale, (a, b)
    # the right-hand side (double-float on the GPU) against the oracle, every entry
    F = torch.tensor(inst["F"], device="cuda")
    Bt = torch.zeros((q, q), dtype=torch.float64, device="cuda")
    h.rhs(F, Bt)
    Bo = rhs(P, inst["F"])
    assert np.abs(Bt.cpu().numpy() - Bo).max() <= 1e-13 * np.abs(Bo).max()
    # FP64 GPU form, then the mixed forms against it
    U64 = torch.zeros((q, q), dtype=torch.float64, device="cuda")
    info64, code64 = h.pcg_solve(F, U64, rtol=1e-10, max_iter=1000, precision="fp64")
    assert code64 == 0
    assert _true_rel(h, F, U64) <= 1.5e-10
    for prec in ("bf16", "tf32", "fp16"):
        U = torch.zeros_like(U64)
        info, code = h.pcg_solve(F, U, rtol=1e-10, max_iter=1000, precision=prec)
        assert code == 0, prec
        assert float(((U - U64).norm() / U64.norm()).item()) <= 1e-8, prec
        assert _true_rel(h, F, U) <= 1.5e-10, prec
    h.close()


def test_rhs_bench_workload(mf):
    """The right-hand side of the bench workload (P2, 2049 x 2049 nodes, 4 instances of
    different seeds, one batched launch) against the oracle, every entry: the double-float
    evaluation is accurate to ~2^-46 of each entry (mass weights only, no cancellation)."""
    import torch
    insts = [metric_instance(n=2049, k=2, seed=s) for s in range(4)]
    h = mf.Handle([i["g1"] for i in insts], [i["g2"] for i in insts], 2, 2049, [1.0] * 4)
    F = torch.tensor(np.stack([i["F"] for i in insts]), device="cuda")
    Bt = torch.zeros((4, h.q, h.q), dtype=torch.float64, device="cuda")
    h.rhs(F, Bt)
    for i, inst in enumerate(insts):
        Bo = rhs(Problem(inst["g1"], inst["g2"], 2, 2049, 1.0), inst["F"])
        assert np.abs(Bt[i].cpu().numpy() - Bo).max() <= 1e-13 * np.abs(Bo).max(), i
    h.close()
