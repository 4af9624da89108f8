"""Seeded synthetic HODLR matrices and right-hand sides.

Memory layout of the returned tensors (the layout the C ABI takes):
* ``D``: shape (2^L, m, m), each block column-major: element (b, i, j) at
  offset b*m*m + j*m + i (strides (m*m, 1, m)).
* ``U``, ``V``: shape (N, r*L), column-major with leading dimension N
  (strides (1, N)); column block j holds the level-(j+1) bases.
* ``B``: shape (N, k), column-major (strides (1, N)).

The synthetic family (the structure of the paper's Sec. 2 HODLR format with
random entries): leaf blocks D_b = G/sqrt(m) + shift*I with G ~ N(0,1), and for
every node alpha at level c the bases U_alpha, V_alpha ~ N(0,1) * 0.5/sqrt(n_c),
n_c = N/2^c the node size. Draw order: D, then U, then V, then B, from one
``torch.Generator`` seeded with ``seed`` on ``device``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch


@dataclass(frozen=True)
class HodlrShape:
    N: int
    L: int
    r: int

    @property
    def m(self) -> int:
        return self.N >> self.L

    @property
    def nleaf(self) -> int:
        return 1 << self.L

    @property
    def rL(self) -> int:
        return self.r * self.L

    def validate(self):
        if self.L < 1 or self.N != self.m << self.L or self.m < 1:
            raise ValueError(f"bad shape {self}")
        if self.r < 1 or self.r > self.m:
            raise ValueError(f"rank must be in 1..m: {self}")


def _colmajor_empty(rows, cols, device, dtype):
    return torch.empty(cols, rows, device=device, dtype=dtype).T


def synthetic_hodlr(shape: HodlrShape, shift: float, seed: int, device="cpu",
                    dtype=torch.float64):
    """Random HODLR operator (D, U, V) of the synthetic family (see module doc)."""
    shape.validate()
    N, L, r, m = shape.N, shape.L, shape.r, shape.m
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    # D: (nleaf, m, m) with column-major blocks
    Dt = torch.randn(shape.nleaf, m, m, generator=g, device=device, dtype=dtype)
    Dt.mul_(1.0 / math.sqrt(m))
    D = Dt.transpose(1, 2)
    idx = torch.arange(m, device=device)
    D[:, idx, idx] += shift
    # U then V: (rL, N) storage viewed as (N, rL) column-major
    scales = torch.tensor([0.5 / math.sqrt(N >> c) for c in range(1, L + 1)],
                          device=device, dtype=dtype).repeat_interleave(r)
    Ut = torch.randn(shape.rL, N, generator=g, device=device, dtype=dtype)
    Ut.mul_(scales[:, None])
    Vt = torch.randn(shape.rL, N, generator=g, device=device, dtype=dtype)
    Vt.mul_(scales[:, None])
    return D, Ut.T, Vt.T, g


def gaussian_rhs(N: int, k: int, generator: torch.Generator, device="cpu",
                 dtype=torch.float64):
    """k right-hand sides b ~ N(0, 1), column-major (N, k)."""
    return torch.randn(k, N, generator=generator, device=device, dtype=dtype).T


def to_math(D, U, V, B=None):
    """numpy float64 copies in the oracle's indexing: D (2^L, m, m) with
    D[b][i, j] = block element (i, j); U, V, B as (rows, cols) arrays."""
    out = [D.detach().cpu().double().numpy().copy(),
           U.detach().cpu().double().numpy().copy(),
           V.detach().cpu().double().numpy().copy()]
    if B is not None:
        out.append(B.detach().cpu().double().numpy().copy())
    return tuple(out)
