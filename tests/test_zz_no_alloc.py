"""GPU test of mofem_precond_noalloc, the allocation-free preconditioner entry point.

Callers that cannot allocate device memory where they apply the preconditioner
(no cudaMalloc/cudaFree and their implicit synchronisation in a latency-critical
loop, or a memory budget held by their own allocator) use this variant; it keeps
its temporaries in a static device array.  The test calls it through the C ABI
twice in a row (the static array keeps the previous call's contents) and checks
each output against the regular mofem_precond(MOFEM_MIXED_BF16) with the BF16
preconditioner tolerance used by the parity tests, then checks that a handle
beyond the static limit is refused.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2109_01173_gb300.inputs import ZERO, SIN_TOP, Profile

pytestmark = pytest.mark.gpu

BF16_PRECOND_TOL = 2.5e-2   # same bound as the BF16 preconditioner parity test


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    torch.cuda.set_device(0)
    import paper_2109_01173_gb300.mofem as mf
    lib = mf.LIB
    lib.mofem_precond_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                          ctypes.c_void_p]
    lib.mofem_precond_noalloc.restype = ctypes.c_int
    return torch, mf, lib


@pytest.mark.parametrize("k,n,dom", [(2, 257, "one"), (1, 301, "two")])
def test_noalloc_matches_precond_two_calls(env, k, n, dom):
    torch, mf, lib = env
    g1, g2 = (ZERO, SIN_TOP) if dom == "one" else (Profile(c2=0.1), Profile(c0=1.0, ca=0.2, cf=1.0))
    h = mf.Handle(g1, g2, k, n, 1.0)
    q = h.q
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        R = torch.tensor(np.random.default_rng(100 + call).standard_normal((q, q)), dtype=torch.float32,
                         device="cuda")
        Z_noalloc = torch.zeros_like(R)
        code = lib.mofem_precond_noalloc(h.h, ctypes.c_void_p(R.data_ptr()), ctypes.c_void_p(Z_noalloc.data_ptr()),
                                         q, stream)
        assert code == mf.OK, lib.mofem_last_error().decode()
        Z_ref = torch.zeros_like(R)
        h.precond(R, Z_ref, "bf16")
        torch.cuda.synchronize()
        rel = float(((Z_noalloc - Z_ref).norm() / Z_ref.norm()).item())
        assert rel <= BF16_PRECOND_TOL, (call, rel)
    h.close()


def test_noalloc_rejects_sizes_beyond_the_static_limit(env):
    torch, mf, lib = env
    h = mf.Handle(ZERO, SIN_TOP, 1, 1025, 1.0)          # q = 1023, ld = 1024: 1047552 > 262144
    R = torch.zeros((h.q, h.q), dtype=torch.float32, device="cuda")
    Z = torch.zeros_like(R)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = lib.mofem_precond_noalloc(h.h, ctypes.c_void_p(R.data_ptr()), ctypes.c_void_p(Z.data_ptr()), h.q, stream)
    assert code == mf.ERR_INVALID_ARG
    assert b"static scratch limit" in lib.mofem_last_error()
    h.close()
