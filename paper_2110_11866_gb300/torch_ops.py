"""torch.autograd wrapper over the C ABI: forward = morlet_forward, backward = morlet_backward.

Marshalling only (tensor checks, output allocation, stream handles); the transform and its adjoint
run in the CUDA library.
"""
from __future__ import annotations

import torch

from . import (MORLET_FP64, morlet_backward, morlet_forward, morlet_plan)


class MorletTransform:
    """Plan plus tensor-level calls for a fixed ragged batch (lengths) and scales (sigmas)."""

    def __init__(self, lengths, sigmas, **kw):
        self.plan = morlet_plan(lengths, sigmas, **kw)
        self.f64 = kw.get("precision", None) == MORLET_FP64
        self.n_in = int(sum(lengths))
        self.n_out = self.n_in * len(sigmas)

    def _check(self, x, dtype):
        if not x.is_cuda or x.dtype != dtype or not x.is_contiguous() or x.numel() != self.n_in:
            raise ValueError(f"expected a contiguous CUDA {dtype} tensor of {self.n_in} samples")

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        self._check(x, torch.float64 if self.f64 else torch.float32)
        W = torch.empty(self.n_out, dtype=torch.complex128 if self.f64 else torch.complex64, device=x.device)
        morlet_forward(self.plan, x, W, torch.cuda.current_stream(x.device))
        return W

    def backward(self, gW: torch.Tensor) -> torch.Tensor:
        gW = gW.contiguous()
        gx = torch.empty(self.n_in, dtype=torch.float64 if self.f64 else torch.float32, device=gW.device)
        morlet_backward(self.plan, gW, gx, torch.cuda.current_stream(gW.device))
        return gx


class MorletFn(torch.autograd.Function):
    """W = MorletFn.apply(x, transform). For a real loss, torch hands backward the gradient
    dLoss/dRe W + i dLoss/dIm W, which is exactly the adjoint's input."""

    @staticmethod
    def forward(ctx, x, transform: MorletTransform):
        ctx.transform = transform
        return transform.forward(x.contiguous())

    @staticmethod
    def backward(ctx, gW):
        return ctx.transform.backward(gW), None
