"""PyTorch autograd front end of the C ABI: the warp and the two losses as
torch.autograd.Function, with gradients for the displacement u only (the
images are data).  Every forward and backward is one call of the library:

* Warp:      J = M o (id + u) (Sec. 2.1, Algorithm gridsampler, forward) by
             reg_warp; its backward g_u = (dJ/dphi) g_J by the sampler
             backward (reg_warp_composite_backward with the identity
             transform).
* LNCCLoss:  C = 1 - S (App. fused LNCC) by reg_loss; the backward recomputes
             the window sums with reg_loss_grad instead of keeping them from
             the forward, so nothing of size N is held between the two.
* MILoss:    C = -MI (Sec. 2.2, App. fused MI), the same way.

The upstream gradient of a loss is a scalar; when it is not 1 the field is
scaled by it (the only arithmetic here besides C = 1 - S on a scalar).
optimize() runs the fused registration loop (reg_run) and returns the field
and its objective history.
"""
from __future__ import annotations

import torch

from . import capi

_IDENTITY = None


def _identity():
    global _IDENTITY
    if _IDENTITY is None:
        _IDENTITY = capi.affine_desc()
    return _IDENTITY


def _scaled(g: torch.Tensor, grad_output: torch.Tensor) -> torch.Tensor:
    if grad_output.numel() == 1 and float(grad_output) == 1.0:
        return g
    return g * grad_output.to(g.dtype)


class Warp(torch.autograd.Function):
    """J = M o (id + u): M [nz, ny, nx] (FP32 / BF16), u [3, nz, ny, nx] FP32 in
    voxels; returns FP32 J.  Differentiable in u."""

    @staticmethod
    def forward(ctx, M, u, pad: int = capi.REG_PAD_BORDER):
        M, u = M.contiguous(), u.contiguous()
        J = capi.reg_warp(M, u, pad)
        ctx.save_for_backward(M, u)
        ctx.pad = pad
        return J

    @staticmethod
    def backward(ctx, gJ):
        M, u = ctx.saved_tensors
        g_u, _ = capi.reg_warp_composite_backward(M, _identity(), gJ.contiguous().float(), u, pad=ctx.pad)
        return None, g_u, None


class _Loss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, F, M, u, loss: capi.RegLossDesc, pad: int):
        F, M, u = F.contiguous(), M.contiguous(), u.contiguous()
        ws = capi.workspace(loss, F)
        sim = capi.reg_loss(loss, F, M, u, ws, pad=pad)
        ctx.save_for_backward(F, M, u)
        ctx.loss, ctx.pad = loss, pad
        value = -sim[0] if loss.kind == capi.REG_LOSS_MI else 1.0 - sim[0]
        return value

    @staticmethod
    def backward(ctx, grad_output):
        F, M, u = ctx.saved_tensors
        ws = capi.workspace(ctx.loss, F)
        _, g = capi.reg_loss_grad(ctx.loss, F, M, u, ws, pad=ctx.pad)
        return None, None, _scaled(g, grad_output), None, None


class LNCCLoss:
    """C = 1 - LNCC(F, M o (id + u)) with a cubic window of side `window`."""

    @staticmethod
    def apply(F, M, u, window: int = 7, eps: float = 1e-9, ants: bool = False, pad: int = capi.REG_PAD_BORDER):
        return _Loss.apply(F, M, u, capi.lncc_desc(window, eps, ants=ants), pad)


class MILoss:
    """C = -MI(F, M o (id + u)), Parzen (cubic B-spline) histogram of `bins`
    bins over the given intensity ranges (default: each image's own)."""

    @staticmethod
    def apply(F, M, u, bins: int = 32, f_range=None, m_range=None, hard: bool = False,
              pad: int = capi.REG_PAD_BORDER):
        fr = f_range if f_range is not None else (float(F.min()), float(F.max()))
        mr = m_range if m_range is not None else (float(M.min()), float(M.max()))
        return _Loss.apply(F, M, u, capi.mi_desc(fr, mr, bins, hard=hard), pad)


def optimize(F, M, cfg, u0=None, iters: int = 200):
    """Register M to F with the fused iteration: returns (u, objective history)."""
    from .register import Registration
    reg = Registration(F, M, cfg, u0=u0)
    res = reg.run(iters)
    return reg.current.clone(), res.objective
