"""GPU parity of heterogeneous batches (problems of different k, n, BC, profile and
gamma solved together by mofem_group_*) against the FP64 oracle, problem by problem,
and the concurrency autotuner (it must restore the initial guesses)."""
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


@pytest.mark.parametrize("prec", ["fp16", "fp64"])
def test_group_solve_vs_oracle(mf, prec):
    import torch
    probs = _problems()
    g = mf.Group(probs)
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
    assert chosen >= 1
    assert all(float(u.abs().max()) == 0.0 for u in U)
    infos, code = g.solve(F, U, rtol=1e-10)
    assert code == 0 and all(i.rel_residual <= 1e-10 for i in infos)
    g.close()
