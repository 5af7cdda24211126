"""Differentiable IMEX Euler heat integration on the MO-PCG solver (Sec. 6).

``HeatIMEX`` is a ``torch.autograd.Function``.  Its forward integrates
u_t - d_u Lap u = f - r u (a nodal source f constant in time and a linear reaction,
both explicit as Sec. 6 treats the reaction term) for ``n_steps`` IMEX Euler steps
from U_0, each step one mixed-precision MO-PCG solve of
(M~ + d_u tau A~) U_{n+1} = (1 - tau r) M~ U_n + tau M~_all f (``mofem_imex_step_src``),
and keeps every ``every``-th state as a checkpoint.  Its backward runs the discrete
adjoint (``mofem_imex_adjoint_step_src``: the same symmetric solve, a mass product,
the f gradient accumulated on the device and the d_u and r inner products), segment
by segment from the last checkpoint, recomputing each segment's states from its
checkpoint, and returns dJ/dU_0, dJ/dd_u, dJ/df and dJ/dr.  All arithmetic runs in
libmofem; this module sequences the calls and holds the checkpoints.

d_u enters the operator (the handle is set up with gamma = 1/(d_u tau)), so a
``HeatSetup`` keeps one handle per d_u value it has seen.
"""
import torch

from . import mofem as mf


class HeatSetup:
    """Domain, discretisation and solver settings of a heat integration.

    ``batch`` independent initial states share d_u and r (the loss is their sum).
    ``rtol`` is the FP64 relative residual of every forward and adjoint solve.
    """

    def __init__(self, g1, g2, k, n, tau, bc=mf.NEUMANN, precision="fp16", rtol=1e-11, batch=1):
        self.g1, self.g2, self.k, self.n, self.tau, self.bc = g1, g2, k, n, float(tau), bc
        self.precision, self.rtol, self.batch = precision, float(rtol), batch
        self._handles = {}
        self.F0 = None

    def handle(self, d_u):
        key = float(d_u)
        h = self._handles.get(key)
        if h is None:
            gam = 1.0 / (key * self.tau)
            B = self.batch
            h = mf.Handle([self.g1] * B, [self.g2] * B, self.k, self.n, [gam] * B, bc=self.bc)
            self._handles[key] = h
            if self.F0 is None:
                self.F0 = torch.zeros((B, self.n, self.n), dtype=torch.float64, device="cuda")
        return h

    def step(self, h, d_u, U, F=None, r=0.0):
        """One forward step from U (B x q x q, FP64, device) with source F (B x n x n or None)."""
        out = torch.empty_like(U)
        h.imex_step_src(float(d_u), self.tau, float(r), U, self.F0 if F is None else F, out, self.rtol,
                        self.precision)
        return out

    def adjoint_step(self, h, d_u, lam, U0, U1, Y=None, r=0.0, dF=None):
        """((1 - tau r) M~ S^{-1} lam, this step's dJ/dd_u, its dJ/dr), dF += tau M~_all^T S^{-1} lam;
        U0, U1 the states before and after the step; Y (in/out) warm-starts the solve from the
        previous step's S^{-1} lam."""
        out = torch.empty_like(lam)
        dd, dr, _, _ = h.imex_adjoint_step_src(float(d_u), self.tau, float(r), lam, U0, U1, out, self.rtol, dF=dF,
                                               precision=self.precision, Y=Y)
        return out, float(sum(dd)), float(sum(dr))

    def close(self):
        for h in self._handles.values():
            h.close()
        self._handles.clear()


class HeatIMEX(torch.autograd.Function):
    """U_N = HeatIMEX.apply(U0, d_u, F, r, setup, n_steps, every).

    U0: (B, q, q) FP64 CUDA tensor; d_u, r: 0-dim tensors; F: (B, n, n) FP64 CUDA tensor
    (nodal source).  Gradients flow to all four.
    """

    @staticmethod
    def forward(ctx, U0, d_u, F, r, setup, n_steps, every):
        du, rr = float(d_u), float(r)
        h = setup.handle(du)
        Fd = F.detach().to(torch.float64).contiguous()
        U = U0.detach().to(torch.float64).contiguous()
        ckpt = [U]
        for i in range(n_steps):
            U = setup.step(h, du, U, Fd, rr)
            if (i + 1) % every == 0 and i + 1 < n_steps:
                ckpt.append(U)
        ctx.setup, ctx.n_steps, ctx.every, ctx.du, ctx.r = setup, n_steps, every, du, rr
        ctx.ckpt, ctx.F = ckpt, Fd
        ctx.meta = (d_u.dtype, d_u.device, r.dtype, r.device)
        return U

    @staticmethod
    def backward(ctx, gU):
        setup, N, M, du, rr = ctx.setup, ctx.n_steps, ctx.every, ctx.du, ctx.r
        h = setup.handle(du)
        lam = gU.detach().to(torch.float64).contiguous()
        Y = torch.zeros_like(lam)   # S^{-1} lam of the previous step: the next solve's initial guess
        gF = torch.zeros_like(ctx.F) if ctx.needs_input_grad[2] else None
        g_du, g_r = 0.0, 0.0
        for s in range(len(ctx.ckpt) - 1, -1, -1):
            start, stop = s * M, min(s * M + M, N)
            states = [ctx.ckpt[s]]
            for _ in range(start, stop):
                states.append(setup.step(h, du, states[-1], ctx.F, rr))
            for n in range(stop - 1, start - 1, -1):
                lam, dd, dr = setup.adjoint_step(h, du, lam, states[n - start], states[n + 1 - start], Y, rr, gF)
                g_du += dd
                g_r += dr
        ctx.ckpt = ctx.F = None
        gu0 = lam if ctx.needs_input_grad[0] else None
        gdu = torch.tensor(g_du, dtype=ctx.meta[0], device=ctx.meta[1]) if ctx.needs_input_grad[1] else None
        gr = torch.tensor(g_r, dtype=ctx.meta[2], device=ctx.meta[3]) if ctx.needs_input_grad[3] else None
        return gu0, gdu, gF, gr, None, None, None


def heat_imex(U0, d_u, setup, n_steps, every=50, F=None, r=None):
    """Differentiable U_N of IMEX Euler (see HeatIMEX); F = None and r = None mean a zero
    source and no reaction (no gradient for them)."""
    if F is None:
        setup.handle(float(d_u))
        F = setup.F0
    if r is None:
        r = torch.zeros((), dtype=torch.float64)
    return HeatIMEX.apply(U0, d_u, F, r, setup, n_steps, every)
