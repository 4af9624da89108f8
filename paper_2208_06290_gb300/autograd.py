"""torch.autograd.Function for  loss = sum_j b_j^T A^{-1} b_j + log|det A|  of a
HODLR matrix A = (D, U_big, V_big): forward and backward both run in libhodlr
(FP64 factor, hodlr_grad); this module only marshals tensors."""
from __future__ import annotations

import torch

from . import binding as hb


class HodlrSolveLogdet(torch.autograd.Function):
    """loss(D, U, V, B) with D (2^L, m, m) column-major blocks, U, V (N, r L) and
    B (N, k) column-major float64 CUDA tensors; L and r are Python ints."""

    @staticmethod
    def forward(ctx, D, U, V, B, L: int, r: int):
        F = hb.hodlr_factor(D, U, V, L, r, "fp64")
        loss, dD, dU, dV, dB = hb.hodlr_grad(F, U, V, B)
        ctx.save_for_backward(dD, dU, dV, dB)
        return torch.tensor(loss, dtype=torch.float64, device=B.device)

    @staticmethod
    def backward(ctx, g):
        dD, dU, dV, dB = ctx.saved_tensors
        return g * dD, g * dU, g * dV, g * dB, None, None


def hodlr_solve_logdet(D, U, V, B, L: int, r: int):
    return HodlrSolveLogdet.apply(D, U, V, B, L, r)
