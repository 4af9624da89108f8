"""torch.autograd.Function for  loss = sum_j b_j^T A^{-1} b_j + log|det A|  of a
HODLR matrix A = (D, U_big, V_big): forward and backward both run in libhodlr;
this module only marshals tensors.

forward: the factorization in the requested precision ("fp64" or "fp32"),
one solve X = A^{-1} B with it, and the factor's log-determinant; the loss is
sum(B * X) + log|det A|. backward (only when a gradient is requested): the
adjoint gradient of hodlr_grad on the same factor (adjoint solves through the
transposed factor, Sec. 3.5), scaled by the incoming gradient.
"""
from __future__ import annotations

import torch

from . import binding as hb


class HodlrSolveLogdet(torch.autograd.Function):
    """loss(D, U, V, B) with D (2^L, m, m) column-major blocks, U, V (N, r L) and
    B (N, k) column-major float64 CUDA tensors; L, r and prec are Python values."""

    @staticmethod
    def forward(ctx, D, U, V, B, L: int, r: int, prec: str = "fp64"):
        if prec not in ("fp64", "fp32"):
            raise ValueError("prec must be 'fp64' or 'fp32'")
        F = hb.hodlr_factor(D, U, V, L, r, prec)
        X = hb.hodlr_solve(F, B.detach().clone())  # clone keeps B's column-major strides
        _, logabsdet = hb.hodlr_logdet(F)
        ctx.F = F
        ctx.save_for_backward(U, V, B)
        return (B * X).sum() + logabsdet

    @staticmethod
    def backward(ctx, g):
        U, V, B = ctx.saved_tensors
        _, dD, dU, dV, dB = hb.hodlr_grad(ctx.F, U, V, B, want_loss=False)
        ctx.F = None
        return g * dD, g * dU, g * dV, g * dB, None, None, None


def hodlr_solve_logdet(D, U, V, B, L: int, r: int, prec: str = "fp64"):
    return HodlrSolveLogdet.apply(D, U, V, B, L, r, prec)
