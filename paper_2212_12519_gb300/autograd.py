"""torch.autograd.Function wrappers whose backward is the hand-written
adjoint kernel (paper Sec. 4: projection layers inside networks such as
unrolled variational networks; Sec. 2.2: matched forward/back pair)."""
from __future__ import annotations

import torch

from . import ops


class JosephTOFLM(torch.autograd.Function):
    """p = A x for TOF listmode events held by ``plan``.

    x: float32 CUDA tensor, one image [n0,n1,n2] shared by all frames or
    [n_frames, n0, n1, n2]; returns p [n_events] in caller order.
    backward: grad_x = A^T grad_p (jp_back_tof_lm)."""

    @staticmethod
    def forward(ctx, x, plan, tof):
        x = x.contiguous()
        ctx.plan, ctx.tof, ctx.shape = plan, tof, x.shape
        return ops.jp_fwd_tof_lm(plan, x, tof)

    @staticmethod
    def backward(ctx, grad_p):
        g = torch.zeros(ctx.shape, dtype=torch.float32, device=grad_p.device)
        ops.jp_back_tof_lm(ctx.plan, grad_p.contiguous(), ctx.tof, g)
        return g, None, None


class JosephNonTOF(torch.autograd.Function):
    """p = A x (non-TOF) for the LORs of ``plan``; backward is jp_back."""

    @staticmethod
    def forward(ctx, x, plan):
        x = x.contiguous()
        ctx.plan, ctx.shape = plan, x.shape
        return ops.jp_fwd(plan, x)

    @staticmethod
    def backward(ctx, grad_p):
        g = torch.zeros(ctx.shape, dtype=torch.float32, device=grad_p.device)
        ops.jp_back(ctx.plan, grad_p.contiguous(), g)
        return g, None


class GaussianResolution(torch.autograd.Function):
    """y = H x, the image-based resolution model (separable Gaussian of
    ``fwhm_mm``, zero outside the grid); backward is H^T = H (symmetric taps)."""

    @staticmethod
    def forward(ctx, x, geom, fwhm_mm, truncate=4.0):
        ctx.geom, ctx.fwhm, ctx.truncate = geom, fwhm_mm, truncate
        return ops.jp_gauss3d(x.contiguous(), geom, fwhm_mm, truncate)

    @staticmethod
    def backward(ctx, g):
        return ops.jp_gauss3d(g.contiguous(), ctx.geom, ctx.fwhm, ctx.truncate), None, None, None


def tof_lm_project(x, plan, tof):
    return JosephTOFLM.apply(x, plan, tof)


def nontof_project(x, plan):
    return JosephNonTOF.apply(x, plan)


class PoissonLogLik(torch.autograd.Function):
    """L = sum_e w_e log(p_e + b_f) for listmode projections p (FP32 compensated sum),
    value and gradient each in one pass of the library's kernels; b holds one
    background per frame of ``plan`` (or one value with plan None)."""

    @staticmethod
    def forward(ctx, p, plan, w, b):
        p = p.contiguous()
        ctx.save_for_backward(p)
        ctx.plan, ctx.w, ctx.b = plan, w, b
        return ops.jp_poisson_loglik_value(plan, p, w, b)

    @staticmethod
    def backward(ctx, gout):
        (p,) = ctx.saved_tensors
        g = ops.jp_poisson_loglik_grad(ctx.plan, p, ctx.w, ctx.b, scale=gout.to(torch.float32).contiguous())
        return g, None, None, None


def poisson_loglik(p, plan, w, b):
    return PoissonLogLik.apply(p, plan, w, b)
