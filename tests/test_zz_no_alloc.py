"""GPU test of mofem_precond_noalloc, the allocation-free preconditioner entry point.

Callers that cannot allocate device memory where they apply the preconditioner
(no cudaMalloc/cudaFree and their implicit synchronisation in a latency-critical
loop, or a memory budget held by their own allocator) use this variant; it keeps
its temporaries in a static device array.  The tests call it through the C ABI:

* twice in a row on one- and multi-instance handles (the static array keeps the
  previous call's contents, of another size in between), each output equal to the
  regular mofem_precond(MOFEM_MIXED_BF16) on the same handle (same BF16 operands,
  same tensor-core tiles, so the same bits) and within the BF16 bound of the FP64
  preconditioner of the same handle;
* on a fresh handle, without the device's free memory changing;
* beyond the static limit, which is refused.

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2109_01173_gb300.inputs import ZERO, SIN_TOP, Profile

pytestmark = pytest.mark.gpu

BF16_PRECOND_TOL = 2.5e-2   # BF16 operands against the FP64 preconditioner (Frobenius, relative)
TWO = (Profile(c2=0.1), Profile(c0=1.0, ca=0.2, cf=1.0))


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


def _noalloc(torch, lib, h, R, Z):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.mofem_precond_noalloc(h.h, ctypes.c_void_p(R.data_ptr()), ctypes.c_void_p(Z.data_ptr()), h.q, stream)


def _check_against_regular(torch, mf, lib, h, seed):
    q, B = h.q, h.batch
    R = torch.tensor(np.random.default_rng(seed).standard_normal((B, q, q)), dtype=torch.float32, device="cuda")
    Z_noalloc = torch.full_like(R, float("nan"))
    assert _noalloc(torch, lib, h, R, Z_noalloc) == mf.OK, lib.mofem_last_error().decode()
    Z_ref = torch.zeros_like(R)
    h.precond(R, Z_ref, "bf16")
    Z64 = torch.zeros((B, q, q), dtype=torch.float64, device="cuda")
    h.precond(R.double(), Z64, "fp64")
    torch.cuda.synchronize()
    assert torch.equal(Z_noalloc, Z_ref), float((Z_noalloc - Z_ref).abs().max())
    for i in range(B):
        rel = float(((Z_noalloc[i].double() - Z64[i]).norm() / Z64[i].norm()).item())
        assert rel <= BF16_PRECOND_TOL, (i, rel)


@pytest.mark.parametrize("k,n,dom", [(2, 257, "one"), (1, 301, "two")])
def test_noalloc_matches_precond_two_calls(env, k, n, dom):
    torch, mf, lib = env
    g1, g2 = (ZERO, SIN_TOP) if dom == "one" else TWO
    h = mf.Handle(g1, g2, k, n, 1.0)
    for call in range(2):
        _check_against_regular(torch, mf, lib, h, 100 + call)
    h.close()


def test_noalloc_batched_instances_two_calls(env):
    """Three instances with their own profiles and gamma (per-instance Q1, lambda and
    s-factors; shared Q2): every instance's Z equals the regular entry point's, on two
    calls in a row, after a call on a larger single-instance handle has left other data
    in the static array."""
    torch, mf, lib = env
    big = mf.Handle(ZERO, SIN_TOP, 2, 257, 1.0)
    _check_against_regular(torch, mf, lib, big, 7)
    big.close()
    tops = [Profile(c0=1.0, sa=a, sf=b) for a, b in ((0.1, 1.0), (0.25, 2.0), (0.3, 3.0))]
    h = mf.Handle([ZERO] * 3, tops, 1, 129, [0.5, 3.0, 9.0])
    assert h.batch * h.q * ((h.q + 63) // 64 * 64) <= 1 << 18
    for call in range(2):
        _check_against_regular(torch, mf, lib, h, 200 + call)
    h.close()


def test_noalloc_call_leaves_free_memory_unchanged(env):
    """After one warm-up call (which may load the module and, with it, the static
    array), a call on a fresh handle changes nothing in the device's free memory: it
    allocates nothing, not even the handle's own BF16 plan."""
    torch, mf, lib = env
    warm = mf.Handle(ZERO, SIN_TOP, 1, 65, 1.0)
    R0 = torch.zeros((warm.q, warm.q), dtype=torch.float32, device="cuda")
    assert _noalloc(torch, lib, warm, R0, torch.zeros_like(R0)) == mf.OK
    torch.cuda.synchronize()
    warm.close()
    h = mf.Handle(*TWO, 2, 201, 2.0)
    R = torch.tensor(np.random.default_rng(5).standard_normal((h.q, h.q)), dtype=torch.float32, device="cuda")
    Z = torch.zeros_like(R)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        assert _noalloc(torch, lib, h, R, Z) == mf.OK
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    assert bool(torch.isfinite(Z).all()) and float(Z.abs().max()) > 0
    h.close()


def test_noalloc_rejects_sizes_beyond_the_static_limit(env):
    torch, mf, lib = env
    h = mf.Handle(ZERO, SIN_TOP, 1, 1025, 1.0)          # q = 1023, ld = 1024: 1047552 > 262144
    R = torch.zeros((h.q, h.q), dtype=torch.float32, device="cuda")
    Z = torch.zeros_like(R)
    assert _noalloc(torch, lib, h, R, Z) == mf.ERR_INVALID_ARG
    assert b"static scratch limit" in lib.mofem_last_error()
    h.close()
