"""PyTorch autograd around the library's forward and adjoint entry points.

``screened_poisson(s, o, alpha)`` is Eq. (1) solved per slice, f = A^{-1}(alpha s + L o) with
A = alpha I + L.  ``correct_stack(I0, alpha, sigma_z)`` is the whole method: s = K_sigma I0
(the truncated anisotropic Gaussian of Sec. 3 "Anisotropic Smoothing") and f = A^{-1}(alpha s +
L I0).  Because A is symmetric, one more solve of the same kind gives lam = A^{-1} dl/df, and
    dl/ds = alpha lam,  dl/do = L lam,  dl/dalpha = <lam, s - f>,
    dl/dI0 = L lam + K^T (alpha lam),  dl/dsigma_z = <alpha lam, (dK/dsigma_z) I0>,
all computed by ``emfuse_backward`` in the library's kernels; these classes only route tensors.

The support floor(3 sigma_z) of the Gaussian is piecewise constant in sigma_z, so dl/dsigma_z
is the derivative with the support held fixed; it does not exist where 3 sigma_z is an
integer (the default sigma_z = 3 is such a point: the derivative there is the one-sided one
from above).

``alpha`` and ``sigma_z`` are 0-dim tensors so that gradient descent can update them; their
values are read on the host for each call.
"""
from __future__ import annotations

import torch

from . import api


def _scalar(x) -> float:
    return float(x.detach().cpu()) if isinstance(x, torch.Tensor) else float(x)


def _like(x, v: float):
    if isinstance(x, torch.Tensor):
        return torch.tensor(v, dtype=x.dtype, device=x.device)
    return None


class ScreenedPoisson(torch.autograd.Function):
    """f = A^{-1}(alpha s + L o) per slice; s, o CUDA float32 [z][y][x]."""

    @staticmethod
    def forward(ctx, s, o, alpha, opts=None):
        a = _scalar(alpha)
        f = api.emfuse_screened_poisson(s.contiguous(), o.contiguous(), a, opts)
        ctx.save_for_backward(s, o, f)
        ctx.alpha_in, ctx.a, ctx.opts = alpha, a, opts
        return f

    @staticmethod
    def backward(ctx, grad_f):
        s, o, f = ctx.saved_tensors
        want = []
        if ctx.needs_input_grad[0]:
            want.append("s")
        if ctx.needs_input_grad[1]:
            want.append("o")
        if ctx.needs_input_grad[2]:
            want.append("alpha")
        if not want:
            return None, None, None, None
        g = api.emfuse_backward(grad_f.contiguous(), f, s, o, 0.0, 0.0, ctx.a, want=tuple(want), opts=ctx.opts)
        return (g.get("s"), g.get("o"),
                _like(ctx.alpha_in, g["alpha"]) if "alpha" in g else None, None)


class CorrectStack(torch.autograd.Function):
    """I2 = A^{-1}(alpha K I0 + L I0) for every slice; I0 CUDA float32 [z][y][x]."""

    @staticmethod
    def forward(ctx, I0, alpha, sigma_z, sigma_xy=1.0, opts=None):
        a, sz = _scalar(alpha), _scalar(sigma_z)
        I0c = I0.contiguous()
        s = api.emfuse_smooth_z(I0c, sigma_xy, sz)
        f = api.emfuse_screened_poisson(s, I0c, a, opts)
        ctx.save_for_backward(I0c, s, f)
        ctx.alpha_in, ctx.sigma_in = alpha, sigma_z
        ctx.a, ctx.sz, ctx.sxy, ctx.opts = a, sz, float(sigma_xy), opts
        return f

    @staticmethod
    def backward(ctx, grad_f):
        I0, s, f = ctx.saved_tensors
        want = []
        if ctx.needs_input_grad[0]:
            want.append("in0")
        if ctx.needs_input_grad[1]:
            want.append("alpha")
        if ctx.needs_input_grad[2]:
            want.append("sigma_z")
        if not want:
            return None, None, None, None, None
        g = api.emfuse_backward(grad_f.contiguous(), f, s, I0, ctx.sxy, ctx.sz, ctx.a, want=tuple(want),
                                opts=ctx.opts)
        return (g.get("in0"),
                _like(ctx.alpha_in, g["alpha"]) if "alpha" in g else None,
                _like(ctx.sigma_in, g["sigma_z"]) if "sigma_z" in g else None, None, None)


def screened_poisson(s, o, alpha, opts=None):
    return ScreenedPoisson.apply(s, o, alpha, opts)


def correct_stack(I0, alpha, sigma_z, sigma_xy: float = 1.0, opts=None):
    return CorrectStack.apply(I0, alpha, sigma_z, sigma_xy, opts)
