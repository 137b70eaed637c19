"""torch.autograd.Function over the C ABI's differentiable functional.

``functional_theta(c, fixer)`` returns (F, theta) of the field held by ``fixer`` (a
GaugeFixer created with ``autograd=True``, FP64-18 storage) after the gauge
transformation g(x) = exp(i sum_a c_a(x) lambda_a); c is a float64 CUDA tensor of shape
(V, 8) in canonical site order.  Forward and backward both run in libgf
(gf_ad_functional / gf_ad_backward); this module only moves pointers.
"""
from __future__ import annotations

import torch

from . import gf


class FunctionalTheta(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c: torch.Tensor, fixer) -> tuple:
        if c.dtype != torch.float64 or not c.is_cuda or not c.is_contiguous() or c.dim() != 2 or c.shape[1] != 8:
            raise ValueError("c must be a contiguous float64 CUDA tensor of shape (V, 8)")
        out = torch.empty(2, dtype=torch.float64, device=c.device)
        gf.gf_ad_functional(fixer.h, c.data_ptr(), out.data_ptr())
        ctx.save_for_backward(c)
        ctx.fixer = fixer
        return out[0], out[1]

    @staticmethod
    def backward(ctx, gF: torch.Tensor, gT: torch.Tensor):
        (c,) = ctx.saved_tensors
        up = torch.stack([gF if gF is not None else torch.zeros((), dtype=torch.float64, device=c.device),
                          gT if gT is not None else torch.zeros((), dtype=torch.float64, device=c.device)])
        up = up.to(dtype=torch.float64).contiguous()
        grad = torch.empty_like(c)
        gf.gf_ad_backward(ctx.fixer.h, c.data_ptr(), up.data_ptr(), grad.data_ptr())
        return grad, None


def functional_theta(c: torch.Tensor, fixer):
    return FunctionalTheta.apply(c, fixer)
