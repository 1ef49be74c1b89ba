"""Differentiation through Frobenius inversion.

:class:`FrobInv` is a ``torch.autograd.Function`` whose forward pass is the
library's ``frob_inv`` and whose backward pass is the library's adjoint
kernel, grad_M = -X^H G X^H (from d(M^{-1}) = -M^{-1} dM M^{-1}).

:func:`sign_newton` runs Newton's iteration for the matrix sign function,
X_{k+1} = (X_k + X_k^{-1}) / 2 (Sec. 5.3 of Dai, Lim and Ye), with every
inverse a Frobenius inversion; with ``checkpoint=True`` each step is wrapped
in ``torch.utils.checkpoint`` so that only the iterates are kept and the
inverses are recomputed in the backward pass.
"""
from __future__ import annotations

import torch
import torch.utils.checkpoint as cp

from . import frob


def _prec_of(m: torch.Tensor) -> str:
    if m.dtype == torch.complex64:
        return "fp32"
    if m.dtype == torch.complex128:
        return "fp64"
    raise TypeError(f"expected complex64 or complex128, got {m.dtype}")


class FrobInv(torch.autograd.Function):
    """X = M^{-1} by Frobenius inversion; backward by the adjoint kernel."""

    @staticmethod
    def forward(ctx, m: torch.Tensor):
        x = frob.frob_inv(m.contiguous(), prec=_prec_of(m)).x
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        (x,) = ctx.saved_tensors
        return frob.inv_adjoint(x, g.contiguous())


def frob_inverse(m: torch.Tensor) -> torch.Tensor:
    """Differentiable M^{-1} (complex64 or complex128, (n, n) or (batch, n, n))."""
    return FrobInv.apply(m)


def _newton_step(x: torch.Tensor) -> torch.Tensor:
    return 0.5 * (x + FrobInv.apply(x))


def sign_newton(m: torch.Tensor, iters: int = 10, checkpoint: bool = True) -> torch.Tensor:
    """`iters` Newton steps for sign(M), each with a Frobenius inversion."""
    x = m
    for _ in range(iters):
        if checkpoint and torch.is_grad_enabled():
            x = cp.checkpoint(_newton_step, x, use_reentrant=False)
        else:
            x = _newton_step(x)
    return x


def sign_loss(m: torch.Tensor, w: torch.Tensor, iters: int = 10, checkpoint: bool = True) -> torch.Tensor:
    """Re tr(W^H sign(M)) summed over the batch."""
    s = sign_newton(m, iters, checkpoint)
    return (w.conj() * s).real.sum()
