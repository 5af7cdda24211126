"""GPU parity of heterogeneous batches (problems of different k, n, BC, profile and
gamma solved together by mofem_group_*) against the FP64 oracle, problem by problem,
in lockstep (one graph and one tensor-core launch per iteration for all groups) and
apart (one stream per group), the two ways bitwise equal; and the autotuner (it must
restore the initial guesses)."""
import numpy as np
import pytest

from oracle.operator import Problem
from oracle import pcg
from paper_2109_01173_gb300.inputs import hetero_instances, fourier_f, Profile, ZERO, SIN_TOP

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mf():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    torch.cuda.set_device(0)
    import paper_2109_01173_gb300.mofem as m
    return m


def _problems():
    probs = hetero_instances(10, n_choices=(17, 25, 33), k_choices=(0, 1, 2, 3, 4), seed=3)
    # two Neumann problems (gamma > 0) and a repeated shape to exercise batching inside a group
    g1 = Profile(c2=0.1)
    probs.append(dict(g1=g1, g2=SIN_TOP, k=2, n=21, gamma=2.0, bc='neumann', F=fourier_f(g1, SIN_TOP, 21, 7)))
    probs.append(dict(g1=g1, g2=SIN_TOP, k=2, n=21, gamma=0.5, bc='neumann', F=fourier_f(g1, SIN_TOP, 21, 8)))
    return probs


@pytest.mark.parametrize("prec,mode", [("fp16", -1), ("bf16", -1), ("tf32", -1), ("fp16", 0), ("fp64", -1)])
def test_group_solve_vs_oracle(mf, prec, mode):
    import torch
    probs = _problems()
    g = mf.Group(probs)
    g.set_mode(mode)
    F = [torch.tensor(p["F"], device="cuda") for p in probs]
    U = [torch.zeros((p["n"] - (2 if p["bc"] == "dirichlet" else 0),) * 2, dtype=torch.float64, device="cuda")
         for p in probs]
    infos, code = g.solve(F, U, rtol=1e-10, max_iter=500, precision=prec)
    assert code == 0
    for p, u in zip(probs, U):
        P = Problem(p["g1"], p["g2"], p["k"], p["n"], p["gamma"], bc=p["bc"])
        Uo, _ = pcg.solve(P, p["F"], rtol=1e-13)
        assert np.linalg.norm(u.cpu().numpy() - Uo) <= 1e-8 * np.linalg.norm(Uo), (p["k"], p["n"], p["bc"])
    g.close()


def test_group_autotune_restores_guesses(mf):
    import torch
    probs = _problems()
    g = mf.Group(probs)
    F = [torch.tensor(p["F"], device="cuda") for p in probs]
    U = [torch.full((p["n"] - (2 if p["bc"] == "dirichlet" else 0),) * 2, 0.0, dtype=torch.float64, device="cuda")
         for p in probs]
    chosen = g.autotune(F, U, rtol=1e-10)
    assert chosen == -1 or chosen >= 1
    assert all(float(u.abs().max()) == 0.0 for u in U)
    infos, code = g.solve(F, U, rtol=1e-10)
    assert code == 0 and all(i.rel_residual <= 1e-10 for i in infos)
    g.close()


def test_group_concurrent_full_size_bitwise(mf):
    """Two groups of full-size problems (P2 and P1, 2049 x 2049 nodes, two instances
    each) solved concurrently on their own streams: their preconditioner GEMM chains
    overlap on the device, and a chain launch that finds another one in flight walks
    its tiles in the dynamic order.  No tile order changes any result (each tile's
    arithmetic and every reduction slot are fixed), so each problem's solution must
    equal bitwise the one from its group's batched handle solved alone."""
    import torch
    from paper_2109_01173_gb300.inputs import metric_instance
    probs = []
    for k in (2, 1):
        for s, gam in ((0, 1.0), (1, 3.0)):
            inst = metric_instance(n=2049, k=k, seed=s, gamma=gam)
            probs.append(dict(g1=inst["g1"], g2=inst["g2"], k=k, n=2049, gamma=gam, bc="dirichlet", F=inst["F"]))
    g = mf.Group(probs)
    F = [torch.tensor(p["F"], device="cuda") for p in probs]
    U = [torch.zeros((2047, 2047), dtype=torch.float64, device="cuda") for _ in probs]
    infos, code = g.solve(F, U, rtol=1e-10, max_iter=500, precision="fp16")
    assert code == 0
    g.close()
    for k, idx in ((2, [0, 1]), (1, [2, 3])):
        h = mf.Handle([probs[i]["g1"] for i in idx], [probs[i]["g2"] for i in idx], k, 2049,
                      [probs[i]["gamma"] for i in idx])
        Ub = torch.zeros((2, 2047, 2047), dtype=torch.float64, device="cuda")
        info, c2 = h.pcg_solve(torch.stack([F[i] for i in idx]), Ub, rtol=1e-10, max_iter=500, precision="fp16")
        assert c2 == 0
        for j, i in enumerate(idx):
            assert torch.equal(Ub[j], U[i]), (k, i)
        h.close()


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_group_lockstep_equals_apart_bitwise(mf, prec):
    """The lockstep form runs each group's arithmetic unchanged (same kernels, same tile
    arithmetic in the shared tensor-core launch, same refinement schedule): every problem's
    solution equals bitwise the one of the groups solved apart."""
    import torch
    probs = _problems()
    g = mf.Group(probs)
    F = [torch.tensor(p["F"], device="cuda") for p in probs]
    out = []
    for mode in (-1, 0):
        g.set_mode(mode)
        U = [torch.zeros((p["n"] - (2 if p["bc"] == "dirichlet" else 0),) * 2, dtype=torch.float64, device="cuda")
             for p in probs]
        infos, code = g.solve(F, U, rtol=1e-10, max_iter=500, precision=prec)
        assert code == 0
        out.append(U)
    for i, (a, b) in enumerate(zip(*out)):
        assert torch.equal(a, b), i
    g.close()
