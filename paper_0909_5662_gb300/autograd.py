"""torch.autograd.Function around the rotation and its hand-written adjoint.

Forward: O'_k = U^T (O_k (x) I_d) U (dmrg_rotate_ops).  Backward: the adjoint
kernels of dmrg_rotate_ops_backward, which recompute what they need from U and
O instead of storing the intermediate product of the forward pass.
"""
from __future__ import annotations

import torch

from .api import dmrg_rotate_ops, dmrg_rotate_ops_backward


class DmrgRotate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, O, d: int, precision: str = "bf16x3"):
        ctx.save_for_backward(U, O)
        ctx.d = d
        ctx.precision = precision
        return dmrg_rotate_ops(U.contiguous(), O.contiguous(), d, precision)

    @staticmethod
    def backward(ctx, G):
        U, O = ctx.saved_tensors
        want_dU = ctx.needs_input_grad[0]
        want_dO = ctx.needs_input_grad[1]
        if not (want_dU or want_dO):
            return None, None, None, None
        G = G.contiguous().to(O.dtype)
        dO, dU = dmrg_rotate_ops_backward(U.contiguous(), O.contiguous(), G, ctx.d, ctx.precision,
                                          want_dO=want_dO, want_dU=want_dU)
        if dO is not None and dO.dtype != O.dtype:
            dO = dO.to(O.dtype)
        return dU, dO, None, None


def rotate(U: torch.Tensor, O: torch.Tensor, d: int, precision: str = "bf16x3") -> torch.Tensor:
    """Differentiable rotation of a batch of block operators."""
    return DmrgRotate.apply(U, O, d, precision)
