"""torch.autograd wrapper of the AKRA 3.0 solve x̂ = (A^T W A + λ_eff I)^{-1} A^T W y (Eq. 14).

Forward: akra_cg_solve.  Backward (λ_eff held fixed), with g = dL/dx̂ (PyTorch's complex
gradient, i.e. dL/dRe + i dL/dIm of every stored component):
    u        = H^{-1} G^{-1} g                     akra_cg_solve_adjoint (implicit adjoint CG)
    dL/dy    = W A u                               akra_apply_A(weighted=True)
    dL/dN^-1 = ω M <A u, y - A x̂>  per pixel        akra_apply_A + akra_weight_grad
Every step runs in libakra.so; this module only marshals tensors.
"""
from __future__ import annotations

import numpy as np
import torch

from . import akra as A


class AkraSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, ninv, plan, prec, tol, maxiter, lam):
        rdt = torch.float32 if prec == A.F32 else torch.float64
        n64 = ninv.detach().to(torch.float64).contiguous()
        A.akra_plan_set_weights(plan, n64, lam)
        yy = y.detach().to(rdt).contiguous()
        if yy.dim() == 2:
            yy = yy[None]
        x, info = A.akra_cg_solve(plan, prec, yy, tol=tol, maxiter=maxiter)
        ctx.plan, ctx.prec, ctx.tol, ctx.maxiter, ctx.lam = plan, prec, tol, maxiter, lam
        ctx.squeeze = y.dim() == 2
        ctx.ydtype, ctx.ndtype = y.dtype, ninv.dtype
        ctx.save_for_backward(yy, n64, x)
        ctx.info = info
        return x[0] if ctx.squeeze else x

    @staticmethod
    def backward(ctx, gx):
        yy, n64, x = ctx.saved_tensors
        plan, prec = ctx.plan, ctx.prec
        op = A.F32 if prec == A.F32 else A.F64
        cdt = torch.complex64 if prec == A.F32 else torch.complex128
        # the plan may have been given other weights since the forward pass
        A.akra_plan_set_weights(plan, n64, ctx.lam)
        g = gx.detach().to(cdt).contiguous()
        if ctx.squeeze:
            g = g[None]
        u, _ = A.akra_cg_solve_adjoint(plan, prec, g, tol=ctx.tol, maxiter=ctx.maxiter)
        uo = u.to(cdt)
        xo = x.to(cdt)
        dy = A.akra_apply_A(plan, op, uo, weighted=True)
        Au = A.akra_apply_A(plan, op, uo)
        Ax = A.akra_apply_A(plan, op, xo)
        dn = A.akra_weight_grad(plan, op, Au, yy, Ax)
        if ctx.squeeze:
            dy = dy[0]
        return dy.to(ctx.ydtype), dn.to(ctx.ndtype), None, None, None, None, None


def akra_solve(y: torch.Tensor, ninv: torch.Tensor, plan, prec: int = A.MIXED, tol: float = 1e-6,
               maxiter: int = 2000, lam: float = 1e-3) -> torch.Tensor:
    """Differentiable x̂(y, N^-1): y [R,2,npix] or [2,npix] shear, ninv [npix] -> complex128
    (complex64 for F32) alm [R,2,ntri] / [2,ntri] of (κ_E, κ_B)."""
    return AkraSolve.apply(y, ninv, plan, prec, tol, maxiter, lam)


def band_power_loss(x: torch.Tensor, lmax: int, edges) -> torch.Tensor:
    """Σ_b mean_{l in (e_b, e_{b+1}]} C_l^E with C_l = [|κ_l0|^2 + 2 Σ_{m>0} |κ_lm|^2]/(2l+1),
    on the E field of a packed alm x [2, ntri] (torch ops; a user-side loss for the tests)."""
    ntri = (lmax + 1) * (lmax + 2) // 2
    ls = np.empty(ntri, np.int64)
    ms = np.empty(ntri, np.int64)
    pos = 0
    for m in range(lmax + 1):
        n = lmax + 1 - m
        ls[pos:pos + n] = np.arange(m, lmax + 1)
        ms[pos:pos + n] = m
        pos += n
    dev = x.device
    l_t = torch.from_numpy(ls).to(dev)
    m0 = torch.from_numpy(ms == 0).to(dev)
    e = x[0]
    p = torch.where(m0, e.real ** 2, 2 * (e.real ** 2 + e.imag ** 2))
    cl = torch.zeros(lmax + 1, dtype=p.dtype, device=dev).index_add_(0, l_t, p)
    cl = cl / (2 * torch.arange(lmax + 1, device=dev, dtype=p.dtype) + 1)
    ell = torch.arange(lmax + 1, device=dev)
    tot = torch.zeros((), dtype=p.dtype, device=dev)
    for b in range(len(edges) - 1):
        sel = (ell > edges[b]) & (ell <= edges[b + 1])
        if bool(sel.any()):
            tot = tot + cl[sel].mean()
    return tot
