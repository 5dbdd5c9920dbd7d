"""Heads as a differentiable function of ln K (adjoint method).

FlowHeads maps a per-cell ln K field (CUDA tensor) to the heads h solving the
steady flow system C(K) h = Q(K).  Its backward pass is one extra AMG-PCG
solve C lambda = dL/dh on the forward pass's hierarchy (C is symmetric) and
the face-flux product kernel gw_adjoint_gradient, which gives dL/dlnK for any
loss L(h) -- e.g. the head misfit at observation cells (gw_misfit), as used in
sensitivity analysis.  Everything runs in libgw's kernels; this module only
passes tensors through the C ABI.
"""
import torch

from . import gw


class FlowHeads(torch.autograd.Function):
    @staticmethod
    def forward(ctx, lnK, nx, ny, nz, bct, bcv, q=None, kz_ratio=1.0, tol=1e-10, maxit=500, opts=None):
        if not lnK.is_cuda or lnK.dtype != torch.float64:
            raise ValueError("lnK must be a float64 CUDA tensor")
        K = torch.exp(lnK.detach())
        Kz = K if kz_ratio == 1.0 else K / kz_ratio
        b = torch.empty_like(K)
        A, _ = gw.gw_assemble(nx, ny, nz, K, K, Kz, bct, bcv, q, b_out=b)
        H = gw.Hierarchy(A, **(opts or {}))
        h, it, rel, st = H.solve(b, tol=tol, maxit=maxit)
        if st != gw.GW_OK:
            raise gw.GwError(st, "forward solve did not converge (relres %.3e after %d iterations)" % (rel, it))
        ctx.save_for_backward(h, K, Kz)
        ctx.H, ctx.grid, ctx.bc, ctx.tol, ctx.maxit = H, (nx, ny, nz), (bct, bcv), tol, maxit
        ctx.forward_iters = it
        return h

    @staticmethod
    def backward(ctx, grad_h):
        h, K, Kz = ctx.saved_tensors
        lam, it, rel, st = ctx.H.solve(grad_h.contiguous(), tol=ctx.tol, maxit=ctx.maxit)
        if st != gw.GW_OK:
            raise gw.GwError(st, "adjoint solve did not converge (relres %.3e after %d iterations)" % (rel, it))
        g = torch.empty_like(h)
        nx, ny, nz = ctx.grid
        gw.gw_adjoint_gradient(nx, ny, nz, K, h, lam, g, Ky=K, Kz=Kz, bct=ctx.bc[0], bcv=ctx.bc[1])
        return (g,) + (None,) * 10


def heads(lnK, nx, ny, nz, bct=(1, 1, 0, 0, 0, 0), bcv=(1.0, 0.0, 0, 0, 0, 0), q=None, kz_ratio=1.0, tol=1e-10,
          maxit=500, **opts):
    """h(lnK), differentiable with respect to lnK."""
    return FlowHeads.apply(lnK, nx, ny, nz, tuple(bct), tuple(bcv), q, kz_ratio, tol, maxit, opts)
