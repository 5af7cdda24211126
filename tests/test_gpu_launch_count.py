"""The solve's kernel-launch count (``mofem_solve_info.kernel_launches``) against the
kernels the CUDA profiling interface saw during the same solve.

Every libmofem kernel is named ``k_*``; the FP64 form's DGEMMs are cuBLAS kernels and
are not part of the count.  Each case runs the solve once untimed (operand copies of
the preconditioner, graph capture) and counts the second solve.
"""
import re

import numpy as np
import pytest

from paper_2109_01173_gb300.inputs import metric_instance

pytestmark = pytest.mark.gpu

OURS = re.compile(r"\bk_[a-z0-9_]+")


@pytest.fixture(scope="module")
def mf():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    torch.cuda.set_device(0)
    # the first profiling session of a process can come back empty (the tracing
    # interface starts lazily): open and close one before any counted solve
    from torch.profiler import profile, ProfilerActivity
    with profile(activities=[ProfilerActivity.CUDA]):
        torch.ones(1024, device="cuda").sum()
        torch.cuda.synchronize()
    import paper_2109_01173_gb300.mofem as m
    return m


def _kernel_names(prof):
    import torch
    out = []
    for e in prof.events():
        if e.device_type != torch.autograd.DeviceType.CUDA:
            continue
        if e.name.startswith("Memcpy") or e.name.startswith("Memset"):
            continue
        out.append(e.name)
    return out


@pytest.mark.parametrize("prec", ["fp16", "bf16", "tf32", "fp64"])
@pytest.mark.parametrize("host_loop", [False, True])
def test_launch_count_matches_profiler(mf, prec, host_loop):
    import torch
    from torch.profiler import profile, ProfilerActivity
    inst = metric_instance(n=257, k=2, seed=3)
    flags = mf.FLAG_HOST_LOOP if host_loop else 0
    h = mf.Handle([inst["g1"]] * 2, [inst["g2"]] * 2, 2, 257, [1.0, 0.5], opts=mf.make_opts(flags=flags))
    F = torch.tensor(np.stack([inst["F"], 0.5 * inst["F"]]), device="cuda")
    U = torch.zeros((2, h.q, h.q), dtype=torch.float64, device="cuda")
    info, code = h.pcg_solve(F, U, rtol=1e-10, max_iter=1000, precision=prec)
    assert code == 0
    U.zero_()
    torch.cuda.synchronize()
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        info, code = h.pcg_solve(F, U, rtol=1e-10, max_iter=1000, precision=prec)
        torch.cuda.synchronize()
    assert code == 0
    names = _kernel_names(prof)
    if not names:
        pytest.skip("the profiler recorded no kernels")
    ours = [n for n in names if OURS.search(n)]
    others = [n for n in names if not OURS.search(n)]
    if prec != "fp64":
        assert not others, sorted(set(others))   # the mixed forms launch libmofem kernels only
    assert len(ours) == info.kernel_launches, (len(ours), info.kernel_launches, info.iterations, info.outer_steps)
    h.close()
