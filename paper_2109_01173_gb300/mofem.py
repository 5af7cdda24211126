"""Thin Python binding of libmofem (ctypes): argument marshalling only.

Every computation happens in libmofem's CUDA kernels behind the C ABI of
``include/mofem.h``; this module converts torch tensors to raw device
pointers and the current torch stream to a ``cudaStream_t``.  There is no CPU
fallback: if ``libmofem.so`` is missing, importing the binding raises.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmofem.so")

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_EIG, ERR_NONFINITE, ERR_BREAKDOWN, ERR_NOT_CONVERGED, ERR_TIMEOUT, \
    ERR_OOM, ERR_UNSUPPORTED = range(10)
DIRICHLET, NEUMANN = 0, 1
FP64, MIXED_TF32, MIXED_BF16, MIXED_FP16 = 0, 1, 2, 3
PENCIL_AVERAGED, PENCIL_DOMINANT, PENCIL_PRODUCT, PENCIL_PARABOLIC, PENCIL_AUA = 0, 1, 2, 3, 4
FLAG_HOST_LOOP, FLAG_FIXED_ITERS, FLAG_TRUE_RESIDUAL = 1, 2, 4

PRECISIONS = {"fp64": FP64, "tf32": MIXED_TF32, "bf16": MIXED_BF16, "fp16": MIXED_FP16}

_GFN = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_double, ctypes.c_void_p)


class Profile(ctypes.Structure):
    _fields_ = [("g", _GFN), ("dg", _GFN), ("ctx", ctypes.c_void_p)]


class Opts(ctypes.Structure):
    _fields_ = [("quad_points", ctypes.c_int), ("pencil", ctypes.c_int), ("max_outer", ctypes.c_int),
                ("inner_rtol", ctypes.c_double), ("flags", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int), ("outer_steps", ctypes.c_int),
                ("batch", ctypes.c_int), ("rel_residual", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("kernel_launches", ctypes.c_longlong)]


class MofemError(RuntimeError):
    def __init__(self, fn, code, lib):
        name = lib.mofem_status_string(code).decode()
        detail = lib.mofem_last_error().decode()
        super().__init__(f"{fn} -> {name}" + (f": {detail}" if detail else ""))
        self.code = code


class ProblemDesc(ctypes.Structure):
    _fields_ = [("g1", Profile), ("g2", Profile), ("k", ctypes.c_int), ("n_nodes", ctypes.c_int),
                ("gamma", ctypes.c_double), ("bc", ctypes.c_int)]


class DibParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("alpha", "gamma", "A1", "A2", "B", "C", "D", "k2", "k3", "d_theta")]


def dib_params(d):
    """mofem_dib_params from a dict with the keys of DibParams."""
    return DibParams(*[float(d[n]) for n, _ in DibParams._fields_])


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libmofem.so not built ({LIB_PATH}); run paper_2109_01173_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    c_int, c_double, vp = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    P = ctypes.POINTER
    sig = {
        "mofem_setup": [P(Profile), P(Profile), c_int, c_int, c_double, c_int, P(Opts), vp, P(vp)],
        "mofem_setup_batched": [c_int, P(Profile), P(Profile), c_int, c_int, P(c_double), c_int, P(Opts), vp, P(vp)],
        "mofem_get_dims": [vp, P(c_int), P(c_int), P(c_int), P(c_int)],
        "mofem_apply": [vp, vp, vp, c_int, c_int, vp],
        "mofem_rhs": [vp, vp, vp, c_int, vp],
        "mofem_precond": [vp, vp, vp, c_int, c_int, vp],
        "mofem_pcg_direction": [vp, vp, vp, P(c_double), P(c_double), vp, vp, c_int, P(c_double), c_int, vp],
        "mofem_pcg_solve": [vp, vp, vp, c_double, c_int, c_int, P(SolveInfo), vp],
        "mofem_imex_step": [vp, c_double, c_double, vp, vp, vp, c_int, P(SolveInfo), vp],
        "mofem_imex_step_tol": [vp, c_double, c_double, vp, vp, vp, c_double, c_int, P(SolveInfo), vp],
        "mofem_rds_step": [vp, c_double, vp, vp, vp, c_double, c_int, P(SolveInfo), vp],
        "mofem_dib_kinetics": [P(DibParams), c_double, vp, vp, vp, vp, ctypes.c_longlong, vp],
        "mofem_dib_equilibrium": [P(DibParams), P(c_double), P(c_double)],
        "mofem_group_layout": [c_int, P(ProblemDesc), P(c_int), P(c_int)],
        "mofem_group_setup": [c_int, P(ProblemDesc), P(Opts), P(vp)],
        "mofem_group_solve": [vp, P(vp), P(vp), c_double, c_int, c_int, P(SolveInfo), vp],
        "mofem_group_autotune": [vp, P(vp), P(vp), c_double, c_int, c_int, P(c_int)],
        "mofem_group_destroy": [vp],
        "mofem_group_set_mode": [vp, c_int],
        "mofem_group_get_tuning": [vp, P(c_int), P(c_int)],
        "mofem_dib_run": [vp, P(DibParams), c_double, c_double, c_int, vp, c_double, c_int, P(c_double),
                          P(SolveInfo), vp],
        "mofem_imex_adjoint_step": [vp, c_double, c_double, vp, vp, vp, vp, P(c_double), c_double, c_int, P(SolveInfo),
                                    vp],
        "mofem_get_eigen": [vp, vp, vp, vp, vp, P(c_int), vp],
        "mofem_imex_step_src": [vp, c_double, c_double, c_double, vp, vp, vp, c_double, c_int, P(SolveInfo), vp],
        "mofem_imex_adjoint_step_src": [vp, c_double, c_double, c_double, vp, vp, vp, vp, vp, vp, P(c_double),
                                        P(c_double), c_double, c_int, P(SolveInfo), vp],
        "mofem_destroy": [vp],
        "mofem_bench_kernel": [vp, c_int, c_int, c_int, vp],
        "mofem_host_tables": [P(Profile), P(Profile), c_int, c_int, c_double, c_int, P(Opts), P(c_int), P(c_int),
                              vp, vp, vp, vp],
        "mofem_host_dd_tables": [P(Profile), P(Profile), c_int, c_int, c_double, c_int, P(Opts), vp, vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = c_int
    lib.mofem_status_string.argtypes = [c_int]
    lib.mofem_status_string.restype = ctypes.c_char_p
    lib.mofem_last_error.argtypes = []
    lib.mofem_last_error.restype = ctypes.c_char_p
    return lib


LIB = _load()

EXPORTED = ["mofem_setup", "mofem_setup_batched", "mofem_get_dims", "mofem_apply", "mofem_rhs", "mofem_precond",
            "mofem_pcg_direction", "mofem_imex_step_tol", "mofem_imex_adjoint_step", "mofem_rds_step",
            "mofem_dib_kinetics", "mofem_dib_run", "mofem_dib_equilibrium", "mofem_group_layout",
            "mofem_group_setup", "mofem_group_solve", "mofem_group_autotune", "mofem_group_destroy",
            "mofem_group_set_mode", "mofem_group_get_tuning",
            "mofem_pcg_solve", "mofem_imex_step", "mofem_destroy", "mofem_status_string", "mofem_last_error",
            "mofem_host_tables", "mofem_host_dd_tables", "mofem_bench_kernel", "mofem_get_eigen",
            "mofem_imex_step_src", "mofem_imex_adjoint_step_src"]


def _check(fn, code):
    if code != OK:
        raise MofemError(fn, code, LIB)


def make_profile(p):
    """C profile from any object with vectorised ``g(x)`` and ``dg(x)`` methods.

    Returns (struct, keepalive); keep ``keepalive`` referenced while the C side may call back.
    """
    g = _GFN(lambda x, ctx: float(p.g(x)))
    dg = _GFN(lambda x, ctx: float(p.dg(x)))
    prof = Profile(g, dg, None)
    return prof, (g, dg)


def make_opts(quad_points=0, pencil=PENCIL_AVERAGED, max_outer=0, inner_rtol=0.0, flags=0):
    return Opts(quad_points, pencil, max_outer, inner_rtol, flags)


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def host_tables(g1, g2, k, n, gamma, bc=DIRICHLET, opts=None):
    """Setup tables computed on the host by the library (no GPU needed)."""
    p1, k1 = make_profile(g1)
    p2, k2 = make_profile(g2)
    d = 1 if k == 0 else k
    P = 2 * d + 1
    q = n - 2 if bc == DIRICHLET else n
    S = np.zeros((8, P, q))
    T = np.zeros((8, P, q))
    Sr = np.zeros((P, q))
    Tr = np.zeros((P, q))
    nt = ctypes.c_int()
    qq = ctypes.c_int()
    o = opts or make_opts()
    code = LIB.mofem_host_tables(ctypes.byref(p1), ctypes.byref(p2), k, n, gamma, bc, ctypes.byref(o),
                                 ctypes.byref(nt), ctypes.byref(qq), S.ctypes.data, T.ctypes.data,
                                 Sr.ctypes.data, Tr.ctypes.data)
    _check("mofem_host_tables", code)
    return dict(n_terms=nt.value, q=qq.value, S=S[:nt.value], T=T[:nt.value], Srh=Sr, Trh=Tr, K=d)


def host_dd_tables(g1, g2, k, n, gamma, bc=DIRICHLET, opts=None):
    """Double-float difference-form tables (hi, lo planes) computed on the host by the
    library: dict(S_hi, S_lo, T_hi, T_lo), each [n_terms][2K+1][q] float32."""
    base = host_tables(g1, g2, k, n, gamma, bc, opts)
    nt, q, P = base["n_terms"], base["q"], 2 * base["K"] + 1
    p1, k1 = make_profile(g1)
    p2, k2 = make_profile(g2)
    S = np.zeros((2, nt, P, q), dtype=np.float32)
    T = np.zeros((2, nt, P, q), dtype=np.float32)
    o = opts or make_opts()
    code = LIB.mofem_host_dd_tables(ctypes.byref(p1), ctypes.byref(p2), k, n, gamma, bc, ctypes.byref(o),
                                    S.ctypes.data, T.ctypes.data)
    _check("mofem_host_dd_tables", code)
    return dict(S_hi=S[0], S_lo=S[1], T_hi=T[0], T_lo=T[1], base=base)


class Handle:
    """One (possibly batched) MO-FEM problem living on the current CUDA device."""

    def __init__(self, g1, g2, k, n, gamma, bc=DIRICHLET, opts=None):
        g1 = g1 if isinstance(g1, (list, tuple)) else [g1]
        g2 = g2 if isinstance(g2, (list, tuple)) else [g2]
        gam = np.atleast_1d(np.asarray(gamma, dtype=np.float64))
        B = max(len(g1), len(g2), gam.size)
        if len(g1) == 1:
            g1 = list(g1) * B
        if len(g2) == 1:
            g2 = list(g2) * B
        if gam.size == 1:
            gam = np.repeat(gam, B)
        keep = []
        arr1 = (Profile * B)()
        arr2 = (Profile * B)()
        for i in range(B):
            arr1[i], k1 = make_profile(g1[i])
            arr2[i], k2 = make_profile(g2[i])
            keep += [k1, k2]
        self._opts = opts or make_opts()
        h = ctypes.c_void_p()
        gam_c = (ctypes.c_double * B)(*gam.tolist())
        code = LIB.mofem_setup_batched(B, arr1, arr2, k, n, gam_c, bc, ctypes.byref(self._opts), _stream(),
                                       ctypes.byref(h))
        _check("mofem_setup_batched", code)
        self.h = h
        self.batch, self.n, self.k, self.bc = B, n, k, bc
        b, nn, q, nt = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check("mofem_get_dims", LIB.mofem_get_dims(h, ctypes.byref(b), ctypes.byref(nn), ctypes.byref(q),
                                                    ctypes.byref(nt)))
        self.q, self.n_terms = q.value, nt.value

    def apply(self, X, Y, precision="fp64", ld=None):
        _check("mofem_apply", LIB.mofem_apply(self.h, _ptr(X), _ptr(Y), ld or X.shape[-1],
                                              PRECISIONS[precision], _stream()))
        return Y

    def rhs(self, F, B, ld=None):
        _check("mofem_rhs", LIB.mofem_rhs(self.h, _ptr(F), _ptr(B), ld or B.shape[-1], _stream()))
        return B

    def precond(self, R, Z, precision="fp64", ld=None):
        _check("mofem_precond", LIB.mofem_precond(self.h, _ptr(R), _ptr(Z), ld or R.shape[-1],
                                                  PRECISIONS[precision], _stream()))
        return Z

    def pcg_direction(self, Z, Qprev, beta, rz, Q, LQ, precision="fp64", ld=None, check=True):
        """Q = Z + beta_i Qprev, LQ = L(Q) and alpha_i = rz_i / <Q, LQ> per instance
        (one search-direction step of MO-PCG).  Returns (alpha list, status code)."""
        n = len(beta)
        arr = ctypes.c_double * n
        b_, r_, a_ = arr(*[float(v) for v in beta]), arr(*[float(v) for v in rz]), arr()
        code = LIB.mofem_pcg_direction(self.h, _ptr(Z), _ptr(Qprev), b_, r_, _ptr(Q), _ptr(LQ),
                                       ld or Z.shape[-1], a_, PRECISIONS[precision], _stream())
        if check:
            _check("mofem_pcg_direction", code)
        return list(a_), code

    def pcg_solve(self, F, U, rtol=1e-10, max_iter=500, precision="bf16", check=True):
        info = SolveInfo()
        code = LIB.mofem_pcg_solve(self.h, _ptr(F), _ptr(U), rtol, max_iter, PRECISIONS[precision],
                                   ctypes.byref(info), _stream())
        if check:
            _check("mofem_pcg_solve", code)
        return info, code

    def imex_step(self, d_u, tau, Un, Fn, Unp1, precision="bf16", check=True):
        info = SolveInfo()
        code = LIB.mofem_imex_step(self.h, d_u, tau, _ptr(Un), _ptr(Fn), _ptr(Unp1), PRECISIONS[precision],
                                   ctypes.byref(info), _stream())
        if check:
            _check("mofem_imex_step", code)
        return info, code

    def imex_step_tol(self, d_u, tau, Un, Fn, Unp1, rtol, precision="fp16", check=True):
        info = SolveInfo()
        code = LIB.mofem_imex_step_tol(self.h, d_u, tau, _ptr(Un), _ptr(Fn), _ptr(Unp1), rtol, PRECISIONS[precision],
                                       ctypes.byref(info), _stream())
        if check:
            _check("mofem_imex_step_tol", code)
        return info, code

    def imex_adjoint_step(self, d_u, tau, Lam1, U1, Lam0, rtol, precision="fp16", check=True, Y=None):
        """Lam0 = M~ S^{-1} Lam1; returns (dJ/dd_u contributions per instance, info, code).
        Y (optional, in/out): initial guess of S^{-1} Lam1, overwritten by it."""
        dd = (ctypes.c_double * self.batch)()
        info = SolveInfo()
        code = LIB.mofem_imex_adjoint_step(self.h, d_u, tau, _ptr(Lam1), _ptr(U1), _ptr(Lam0),
                                           _ptr(Y) if Y is not None else None, dd, rtol,
                                           PRECISIONS[precision], ctypes.byref(info), _stream())
        if check:
            _check("mofem_imex_adjoint_step", code)
        return list(dd), info, code

    def imex_step_src(self, d_u, tau, r, Un, F, Unp1, rtol, precision="fp16", check=True):
        """U_np1 from (M~ + d_u tau A~) U_np1 = (1 - tau r) M~ U_n + tau M~_all F."""
        info = SolveInfo()
        code = LIB.mofem_imex_step_src(self.h, d_u, tau, r, _ptr(Un), _ptr(F), _ptr(Unp1), rtol,
                                       PRECISIONS[precision], ctypes.byref(info), _stream())
        if check:
            _check("mofem_imex_step_src", code)
        return info, code

    def imex_adjoint_step_src(self, d_u, tau, r, Lam1, U0, U1, Lam0, rtol, dF=None, precision="fp16", check=True,
                              Y=None):
        """Lam0 = (1 - tau r) M~ S^{-1} Lam1, dF += tau M~_all^T S^{-1} Lam1 (if given); returns
        (dJ/dd_u and dJ/dr contributions per instance, info, code)."""
        dd = (ctypes.c_double * self.batch)()
        dr = (ctypes.c_double * self.batch)()
        info = SolveInfo()
        code = LIB.mofem_imex_adjoint_step_src(self.h, d_u, tau, r, _ptr(Lam1), _ptr(U0), _ptr(U1), _ptr(Lam0),
                                               _ptr(Y) if Y is not None else None,
                                               _ptr(dF) if dF is not None else None, dd, dr, rtol,
                                               PRECISIONS[precision], ctypes.byref(info), _stream())
        if check:
            _check("mofem_imex_adjoint_step_src", code)
        return list(dd), list(dr), info, code

    def rds_step(self, tau, Un, Fn, Unp1, rtol=0.0, precision="fp16", check=True):
        info = SolveInfo()
        code = LIB.mofem_rds_step(self.h, tau, _ptr(Un), _ptr(Fn), _ptr(Unp1), rtol, PRECISIONS[precision],
                                  ctypes.byref(info), _stream())
        if check:
            _check("mofem_rds_step", code)
        return info, code

    def dib_run(self, params, rho, tau, n_steps, U, rtol=0.0, precision="fp16", increments=False, check=True):
        """n_steps of the DIB model on U = [eta; theta] in place; returns (info, code, increments or None)."""
        info = SolveInfo()
        inc = (ctypes.c_double * max(n_steps, 1))() if increments else None
        p = dib_params(params)
        code = LIB.mofem_dib_run(self.h, ctypes.byref(p), rho, tau, n_steps, _ptr(U), rtol, PRECISIONS[precision],
                                 inc, ctypes.byref(info), _stream())
        if check:
            _check("mofem_dib_run", code)
        return info, code, (list(inc)[:n_steps] if increments else None)

    def eigen(self):
        """Preconditioner eigen data as FP64 device tensors (Q1 [batch][q][q], Q2 [q][q],
        lambda [batch][q], mu [q]) and whether the divisor is lambda_a mu_b (True) or
        lambda_a + mu_b (False)."""
        import torch
        q, B = self.q, self.batch
        Q1 = torch.empty((B, q, q), dtype=torch.float64, device="cuda")
        Q2 = torch.empty((q, q), dtype=torch.float64, device="cuda")
        lam = torch.empty((B, q), dtype=torch.float64, device="cuda")
        mu = torch.empty((q,), dtype=torch.float64, device="cuda")
        prod = ctypes.c_int()
        _check("mofem_get_eigen", LIB.mofem_get_eigen(self.h, _ptr(Q1), _ptr(Q2), _ptr(lam), _ptr(mu),
                                                      ctypes.byref(prod), _stream()))
        return Q1, Q2, lam, mu, bool(prod.value)

    def bench_kernel(self, kernel, precision="bf16", reps=1):
        """Launch one hot kernel `reps` times on internal buffers (timing hook)."""
        _check("mofem_bench_kernel", LIB.mofem_bench_kernel(self.h, kernel, PRECISIONS[precision], reps, _stream()))

    def close(self):
        if self.h:
            LIB.mofem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dib_kinetics(params, rho, eta, theta, f, g):
    """f = rho f(eta, theta), g = rho g(eta, theta) elementwise on device tensors."""
    p = dib_params(params)
    _check("mofem_dib_kinetics", LIB.mofem_dib_kinetics(ctypes.byref(p), rho, _ptr(eta), _ptr(theta), _ptr(f),
                                                         _ptr(g), eta.numel(), _stream()))


def dib_equilibrium(params):
    """(eta_e, theta_e): zero of the DIB kinetics (host Newton in libmofem)."""
    p = dib_params(params)
    e, t = ctypes.c_double(), ctypes.c_double()
    _check("mofem_dib_equilibrium", LIB.mofem_dib_equilibrium(ctypes.byref(p), ctypes.byref(e), ctypes.byref(t)))
    return e.value, t.value


def _problem_array(problems):
    """ctypes array of problem descriptors from dicts with g1, g2, k, n, gamma, bc ('dirichlet'/'neumann')."""
    arr = (ProblemDesc * len(problems))()
    keep = []
    for i, d in enumerate(problems):
        p1, k1 = make_profile(d["g1"])
        p2, k2 = make_profile(d["g2"])
        keep += [k1, k2]
        bc = d.get("bc", DIRICHLET)
        bc = {"dirichlet": DIRICHLET, "neumann": NEUMANN}.get(bc, bc)
        arr[i] = ProblemDesc(p1, p2, int(d["k"]), int(d["n"]), float(d["gamma"]), int(bc))
    return arr, keep


def group_layout(problems):
    """(number of groups, group index of each problem), computed on the host."""
    arr, keep = _problem_array(problems)
    ng = ctypes.c_int()
    of = (ctypes.c_int * len(problems))()
    _check("mofem_group_layout", LIB.mofem_group_layout(len(problems), arr, ctypes.byref(ng), of))
    return ng.value, list(of)


class Group:
    """Heterogeneous batch of elliptic problems (see mofem_group_setup)."""

    def __init__(self, problems, opts=None):
        arr, keep = _problem_array(problems)
        self.count = len(problems)
        self.g = ctypes.c_void_p()
        _check("mofem_group_setup", LIB.mofem_group_setup(self.count, arr, ctypes.byref(opts) if opts else None,
                                                          ctypes.byref(self.g)))

    def _ptrs(self, tensors):
        return (ctypes.c_void_p * self.count)(*[_ptr(t) for t in tensors])

    def solve(self, F, U, rtol=1e-10, max_iter=500, precision="fp16", check=True):
        infos = (SolveInfo * self.count)()
        code = LIB.mofem_group_solve(self.g, self._ptrs(F), self._ptrs(U), rtol, max_iter, PRECISIONS[precision],
                                     infos, _stream())
        if check:
            _check("mofem_group_solve", code)
        return list(infos), code

    def set_mode(self, mode):
        """-1: lockstep (one graph, one tensor-core launch per iteration for all groups);
        0: groups apart, all in flight; m > 0: apart, m in flight."""
        _check("mofem_group_set_mode", LIB.mofem_group_set_mode(self.g, int(mode)))

    def tuning(self):
        """(mode, operator-apply tile divisor) the later solves use."""
        m, d = ctypes.c_int(), ctypes.c_int()
        _check("mofem_group_get_tuning", LIB.mofem_group_get_tuning(self.g, ctypes.byref(m), ctypes.byref(d)))
        return m.value, d.value

    def autotune(self, F, U, rtol=1e-10, max_iter=500, precision="fp16"):
        chosen = ctypes.c_int()
        _check("mofem_group_autotune", LIB.mofem_group_autotune(self.g, self._ptrs(F), self._ptrs(U), rtol, max_iter,
                                                                PRECISIONS[precision], ctypes.byref(chosen)))
        return chosen.value

    def close(self):
        if self.g:
            LIB.mofem_group_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
