"""Operation and byte counts of the HODLR factor / solve / matvec (Sec. 3.4).

Flop counts are the exact multiply-add counts of Alg. 1 / Alg. 2 summed in
closed form (the paper's Theorem t_f approximates the level term by
2 r^2 N (L + L^2); the loop over child levels c = 1..L touches c-1 ancestor
blocks, which gives 2 r^2 N L^2, plus the 2r x 2r coupling LUs and solves).
These are the algorithmic counts used for TFLOP/s, whatever the kernels
actually execute.
"""
from __future__ import annotations


def factor_flops(N: int, m: int, r: int, L: int) -> float:
    leaf = 2.0 / 3.0 * m * m * N + 2.0 * m * r * N * L
    panels = 2.0 * r * r * N * L * L
    coupling = sum((1 << (c - 1)) * (2.0 / 3.0 * (2 * r) ** 3 + 8.0 * r ** 3 * (c - 1)) for c in range(1, L + 1))
    return leaf + panels + coupling


def solve_flops(N: int, m: int, r: int, L: int, k: int = 1) -> float:
    return k * (2.0 * m * N + 4.0 * r * N * L + 8.0 * r * r * ((1 << L) - 1))


def matvec_flops(N: int, m: int, r: int, L: int, k: int = 1) -> float:
    return k * (2.0 * m * N + 4.0 * r * N * L)


def storage_elems(N: int, m: int, r: int, L: int) -> int:
    """Entries of the HODLR matrix: mN + 2rNL (Sec. 3.4 bullets)."""
    return m * N + 2 * r * N * L


def matvec_bytes(N: int, m: int, r: int, L: int, k: int = 1) -> float:
    """Compulsory FP64 bytes of Y = A X: D, U, V once, X read once per level
    pass (L+1 passes) and Y written once and updated L times (read+write)."""
    return 8.0 * (storage_elems(N, m, r, L) + N * k * (L + 1) + N * k * (2 * L + 1))


def update_bytes(N: int, r: int, c: int, ncols: int, elem: int) -> float:
    """Algorithmic bytes of one level's ancestor update R(:, 0:ncols) -= Y_own W:
    R read and written once, the own block Y(:, c-1) read once (W is small)."""
    return float(elem) * N * (2 * ncols + r)


def project_bytes(N: int, r: int, ncols: int, elem: int) -> float:
    """Algorithmic bytes of one level's projection V^T R(:, 0:ncols): R and the
    level's V block read once."""
    return float(elem) * N * (ncols + r)


def solve_bytes(N: int, m: int, r: int, L: int, k: int, prec: str) -> float:
    """Compulsory bytes of one k-column solve (or adjoint solve) with a factor
    of precision `prec`: the factor read once (leaf inverses or LUs, Y_big and
    the level's V blocks, the 2r x 2r coupling inverses in FP64) and the k
    right-hand sides read and written once per level (in FP32 for a
    low-precision factor, FP64 otherwise)."""
    e_leaf = 8 if prec == "fp64" else 4
    e_panel = {"fp64": 8, "fp32": 4}.get(prec, 2)
    e_x = 8 if prec == "fp64" else 4
    factor = e_leaf * N * m + 2.0 * e_panel * N * r * L + 8.0 * 4 * r * r * ((1 << L) - 1)
    return factor + 2.0 * e_x * N * k * L
