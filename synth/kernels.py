"""Seeded kernel-matrix and boundary-integral HODLR inputs (untimed construction).

The solver's input is the HODLR operator (D, U_big, V_big). These generators
build it from a dense matrix that is never formed: leaf blocks are evaluated
exactly, and every off-diagonal sibling block A(I_alpha, I_beta) is compressed
to the fixed rank r by a randomized SVD (range finder with one power
iteration, Gaussian test matrix, oversampling 10), every block of every size
evaluated tile by tile. The compression error is not part of the solver's
problem: the oracle and the GPU path both take the generated (D, U, V) as the
matrix; ``stats`` (when given a dict) receives, per level, an estimate of the
relative compression error of the level's first blocks.

Workloads (structure of the paper's Sec. 4 experiments; real field):
* ``bie_hodlr``: 2D Laplace double-layer second-kind BIE on the star curve
  rho(t) = 1 + 0.3 cos 5t, trapezoid rule on N equispaced parameters, natural
  curve order, A = -1/2 I + D with D(x_i, y_j) w_j off the diagonal,
  d(x, y) = n(y).(x - y) / (2 pi |x - y|^2), n the outward normal, and the
  smooth-quadrature diagonal -1/2 - w_i kappa_i / (4 pi) (the limit of the
  kernel at x = y, kappa the curvature). Gauss's identity gives A 1 = -1 up to
  quadrature error.
* ``kernel_hodlr``: symmetric kernel matrices on points uniform in [0,1]^d
  ordered by a kd-tree of median splits (axes cycling with depth, leaves of
  m points), K(x, y) = k(|x - y|) + nugget * delta; the symmetric split of
  each block's SVD gives U = V.
"""
from __future__ import annotations

import math
import os
import sys
import time

import torch

_VERBOSE = os.environ.get("HODLR_SYNTH_VERBOSE", "") not in ("", "0")


def _log(msg):
    if _VERBOSE:
        sys.stderr.write(f"[synth] {msg}\n")

from .generators import HodlrShape


# ------------------------------------------------------------------ geometry
def star_curve(N: int, device="cpu", dtype=torch.float64):
    """Points, outward unit normals, trapezoid weights and curvature on the
    star curve rho(t) = 1 + 0.3 cos(5t), t_i = 2 pi i / N."""
    t = torch.arange(N, device=device, dtype=dtype) * (2 * math.pi / N)
    rho = 1 + 0.3 * torch.cos(5 * t)
    drho = -1.5 * torch.sin(5 * t)
    ddrho = -7.5 * torch.cos(5 * t)
    c, s = torch.cos(t), torch.sin(t)
    x = torch.stack([rho * c, rho * s], dim=1)
    tx = drho * c - rho * s
    ty = drho * s + rho * c
    speed = torch.sqrt(tx * tx + ty * ty)
    normal = torch.stack([ty / speed, -tx / speed], dim=1)  # outward for a counter-clockwise curve
    w = speed * (2 * math.pi / N)
    kappa = (rho * rho + 2 * drho * drho - rho * ddrho) / (rho * rho + drho * drho) ** 1.5
    return x, normal, w, kappa


def bie_block(x, normal, w, rows, cols):
    """Off-diagonal entries A(rows, cols) = d(x_i, y_j) w_j (no i == j)."""
    xi = x[rows]  # (..., a, 2)
    yj = x[cols]  # (..., b, 2)
    d = xi.unsqueeze(-2) - yj.unsqueeze(-3)
    r2 = (d * d).sum(-1)
    nd = (d * normal[cols].unsqueeze(-3)).sum(-1)
    return nd / (2 * math.pi * r2) * w[cols].unsqueeze(-2)


def bie_dense(N: int, dtype=torch.float64):
    """The full N x N BIE matrix (small N only, for checks)."""
    x, n, w, kappa = star_curve(N, dtype=dtype)
    idx = torch.arange(N)
    A = torch.zeros(N, N, dtype=dtype)
    off = idx[:, None] != idx[None, :]
    blk = bie_block(x, n, w, idx, idx)
    A[off] = blk[off]
    A[idx, idx] = -0.5 - w * kappa / (4 * math.pi)
    return A


def kd_order(pts: torch.Tensor, m: int) -> torch.Tensor:
    """Permutation ordering the points by a kd-tree of median splits, axes
    cycling with depth, until nodes hold m points (N = m 2^L); stable sorts."""
    N, dim = pts.shape
    perm = torch.arange(N, device=pts.device)
    size = N
    depth = 0
    while size > m:
        axis = depth % dim
        groups = perm.view(-1, size)
        keys = pts[groups, axis]
        order = torch.argsort(keys, dim=1, stable=True)
        perm = torch.gather(groups, 1, order).reshape(-1)
        size //= 2
        depth += 1
    return perm


# ------------------------------------------------------------------ compression
def _orth(Y, rtol=1e-13):
    """(Q, R) with Y ~= Q R and Q's columns orthonormal, spanning the
    numerically significant range of each (tall) matrix of the batch: the
    Gram matrix Y^T Y is formed by a device matmul in FP64, its (small)
    eigendecomposition is done on the CPU, Q = Y E diag(lambda)^{-1/2} on the
    device; directions with lambda <= rtol * lambda_max are dropped (their
    columns of Q are zero). Only matmuls and elementwise operations run on
    the device."""
    Yd = Y.double()
    G = (Yd.transpose(1, 2) @ Yd).cpu()
    lam, E = torch.linalg.eigh(G)
    keep = lam > rtol * lam[:, -1:].clamp(min=1e-300)
    inv_sqrt = torch.where(keep, lam.clamp(min=1e-300).rsqrt(), torch.zeros_like(lam))
    sq = torch.where(keep, lam.clamp(min=0).sqrt(), torch.zeros_like(lam))
    Q = (Yd @ (E * inv_sqrt[:, None, :]).to(Y.device)).to(Y.dtype)
    R = (sq[:, :, None] * E.transpose(1, 2))                      # CPU, FP64
    return Q, R


def _qr(Y):
    return _orth(Y)[0]


def _core_split(Bt, r, rtol=1e-14):
    """Rank-r split of the small wide cores B = Bt^T (p x n, p = r + oversampling):
    with B B^T = E diag(lambda) E^T (FP64 Gram matrix formed on the device,
    eigendecomposed on the CPU), the left factor E_r diag(sigma_r)^(1/2) and
    the right factor B^T E_r diag(sigma_r)^(-1/2), sigma = lambda^(1/2), for
    the r largest lambda; their product E_r E_r^T B is B projected on its
    dominant left singular subspace, as the truncated SVD gives. Directions
    with lambda <= rtol * lambda_max (below the Gram matrix's resolution) get
    zero columns. Cores of very low rank have many zero rows (directions the
    range finder dropped); the eigensolver takes them as they are, unlike
    some LAPACK builds' SVD."""
    Bd = Bt.double()
    G = (Bd.transpose(1, 2) @ Bd).cpu()
    lam, E = torch.linalg.eigh(G)                         # ascending
    lam = lam[:, -r:].flip(-1)
    E = E[:, :, -r:].flip(-1)
    keep = lam > rtol * lam[:, :1].clamp(min=1e-300)
    q = torch.where(keep, lam.clamp(min=1e-300) ** 0.25, torch.zeros_like(lam))   # sigma^(1/2)
    qinv = torch.where(keep, 1.0 / q.clamp(min=1e-300), torch.zeros_like(lam))
    left = (E * q[:, None, :]).to(Bt.device, Bt.dtype)       # p x r
    right = (E * qinv[:, None, :]).to(Bt.device)             # p x r, applied to B^T below
    return left, (Bd @ right).to(Bt.dtype)


def _rsvd_blocks(entries, row_start, col_start, n, r, g, device, oversample=10, budget=1 << 27):
    """Randomized range finder with one power iteration on blocks
    K_b = A(row_start[b] + [0, n), col_start[b] + [0, n)), evaluated tile by
    tile. Returns (Ub, Vb) with K_b ~= Ub[b] Vb[b]^T, rank r."""
    nblk = row_start.numel()
    p = r + oversample
    if n * n <= budget:
        bs, tr = max(1, budget // (n * n)), n
    else:
        bs, tr = 1, max(1, budget // n)
    Uo = torch.empty(nblk, n, r, device=device)
    Vo = torch.empty(nblk, n, r, device=device)
    ar = torch.arange(n, device=device)
    for b0 in range(0, nblk, bs):
        b1 = min(nblk, b0 + bs)
        nb = b1 - b0
        cols = col_start[b0:b1, None] + ar[None, :]

        def tile(r0, r1):
            return entries(row_start[b0:b1, None] + ar[None, r0:r1], cols)

        def times(M):      # block @ M
            out = torch.empty(nb, n, M.shape[-1], device=device)
            for r0 in range(0, n, tr):
                r1 = min(n, r0 + tr)
                out[:, r0:r1] = tile(r0, r1) @ M
            return out

        def ttimes(M):     # block^T @ M
            out = torch.zeros(nb, n, M.shape[-1], device=device)
            for r0 in range(0, n, tr):
                r1 = min(n, r0 + tr)
                out += tile(r0, r1).transpose(1, 2) @ M[:, r0:r1]
            return out

        Om = torch.randn(nb, n, p, generator=g, device=device)
        Q = _qr(times(Om))
        Q = _qr(times(_qr(ttimes(Q))))
        Bt = ttimes(Q)                                  # block^T Q = B^T
        left, right = _core_split(Bt, r)
        Uo[b0:b1] = Q @ left
        Vo[b0:b1] = right
    return Uo, Vo


def compress_blocks(entries, row_start, col_start, n, r, g, device):
    """Rank-r factors of the n x n blocks at (row_start[b], col_start[b]) by
    the randomized SVD (Gaussian test matrix, oversampling 10, one power
    iteration), at every block size."""
    return _rsvd_blocks(entries, row_start, col_start, n, r, g, device)


def compression_error(entries, row_start, col_start, n, Ub, Vb, g, device, nprobe=4, budget=1 << 27):
    """Relative error |(K - U V^T) w| / |K w| of the first blocks' rank-r
    factors along nprobe Gaussian vectors w, blocks evaluated tile by tile
    (an estimate of the spectral-norm error, for the record)."""
    nb = min(int(row_start.numel()), 4)
    ar = torch.arange(n, device=device)
    tr = max(1, budget // max(n, 1))
    errs = []
    for b in range(nb):
        w = torch.randn(n, nprobe, generator=g, device=device)
        kw = torch.empty(n, nprobe, device=device)
        for r0 in range(0, n, tr):
            r1 = min(n, r0 + tr)
            blk = entries((row_start[b] + ar[r0:r1])[None, :], (col_start[b] + ar)[None, :])[0]
            kw[r0:r1] = blk @ w
        uv = Ub[b] @ (Vb[b].T @ w)
        errs.append(float((kw - uv).norm() / kw.norm().clamp(min=1e-300)))
    return max(errs) if errs else 0.0


def _assemble(shape: HodlrShape, leaf_fn, entries, seed, device, symmetric, stats=None):
    """D (column-major blocks), U, V (column-major N x rL) in FP64."""
    N, L, r, m = shape.N, shape.L, shape.r, shape.m
    g = torch.Generator(device=device)
    g.manual_seed(seed + 1000)
    ge = torch.Generator(device=device)  # probes of the error estimates (leaves g's draws unchanged)
    ge.manual_seed(seed + 2000)
    if stats is not None:
        stats.setdefault("compression_rel_err", {})
    Dt = torch.empty(shape.nleaf, m, m, device=device, dtype=torch.float64)
    step = max(1, (1 << 26) // (m * m))
    for b0 in range(0, shape.nleaf, step):
        b1 = min(shape.nleaf, b0 + step)
        Dt[b0:b1] = leaf_fn(b0, b1).transpose(1, 2).double()
    D = Dt.transpose(1, 2)
    Ut = torch.empty(shape.rL, N, device=device, dtype=torch.float64)
    Vt = torch.empty(shape.rL, N, device=device, dtype=torch.float64)
    for c in range(1, L + 1):
        n = N >> c
        t0 = time.time()
        cols = slice((c - 1) * r, c * r)
        if symmetric:
            # blocks A(I_left, I_right) of the 2^(c-1) pairs; U = V by the symmetric split
            j = torch.arange(1 << (c - 1), device=device)
            Ub, Vb = compress_blocks(entries, 2 * j * n, (2 * j + 1) * n, n, r, g, device)
            if stats is not None:
                stats["compression_rel_err"][c] = compression_error(entries, 2 * j * n, (2 * j + 1) * n, n, Ub, Vb,
                                                                    ge, device)
            for jj in range(1 << (c - 1)):
                Ut[cols, (2 * jj) * n:(2 * jj + 1) * n] = Ub[jj].T.double()
                Ut[cols, (2 * jj + 1) * n:(2 * jj + 2) * n] = Vb[jj].T.double()
            Vt[cols] = Ut[cols]
        else:
            # block b < 2^c: rows of node b, columns of its sibling b ^ 1
            b = torch.arange(1 << c, device=device)
            Ub, Vb = compress_blocks(entries, b * n, (b ^ 1) * n, n, r, g, device)
            if stats is not None:
                stats["compression_rel_err"][c] = compression_error(entries, b * n, (b ^ 1) * n, n, Ub, Vb, ge,
                                                                    device)
            Ut[cols] = Ub.transpose(1, 2).permute(1, 0, 2).reshape(r, N).double()
            Vt[cols] = Vb[b ^ 1].transpose(1, 2).permute(1, 0, 2).reshape(r, N).double()
        if _VERBOSE:
            if Ut.is_cuda:
                torch.cuda.synchronize()
            _log(f"level {c}: blocks of {n} rows in {time.time() - t0:.2f} s")
    return D, Ut.T, Vt.T


def bie_offdiag_entries(N: int, device="cpu"):
    """Evaluator entries(rows, cols) -> FP32 (batch, a, b) of the BIE's
    off-diagonal entries A(rows, cols), for index tensors rows (batch, a) and
    cols (batch, b) that are contiguous, disjoint index ranges per batch entry
    (the sibling blocks the compression evaluates tile by tile).

    For nearby points n(y).(x - y) is second order in the distance while
    x - y is first order. Entries whose curve-order distance is below
    `band` = max(256, N / 128) come from the FP64 geometry; the others from
    x - y formed in FP64 and the rest in FP32 (error relative to the block's
    largest entry about 1.2e-7 / (kappa |x - y|), <= 1.1e-6 beyond the band at
    N = 2^16; from FP32 coordinates it would be ~1.6e-7 / (kappa |x - y|^2),
    the whole entry for neighbours)."""
    x, nrm, w, _ = star_curve(N, device=device, dtype=torch.float64)
    n32, w32 = nrm.float(), w.float()
    band = max(256, N // 128)

    def entries(rows, cols):
        b = cols.shape[-1]
        if 2 * band >= b:
            return bie_block(x, nrm, w, rows, cols).float()
        dx = (x[rows, 0][..., :, None] - x[cols, 0][..., None, :]).float()
        dy = (x[rows, 1][..., :, None] - x[cols, 1][..., None, :]).float()
        nd = dx * n32[cols, 0][..., None, :] + dy * n32[cols, 1][..., None, :]
        out = nd / ((2 * math.pi) * (dx * dx + dy * dy)) * w32[cols][..., None, :]
        lo, hi = rows[:, :1], rows[:, -1:]
        dist = torch.minimum(torch.remainder(cols - hi, N), torch.remainder(lo - cols, N))
        e, j = (dist < band).nonzero(as_tuple=True)
        if e.numel():
            out[e, :, j] = bie_block(x, nrm, w, rows[e], cols[e, j][:, None])[..., 0].float()
        return out

    return entries


def bie_hodlr(shape: HodlrShape, device="cpu", seed=2, stats=None):
    """HODLR operator of the star-curve Laplace BIE (see module doc)."""
    shape.validate()
    N, m = shape.N, shape.m
    x, nrm, w, kappa = star_curve(N, device=device, dtype=torch.float64)
    diag = (-0.5 - w * kappa / (4 * math.pi))

    def leaf_fn(b0, b1):
        idx = torch.arange(b0 * m, b1 * m, device=device).view(b1 - b0, m)
        blk = bie_block(x, nrm, w, idx, idx)
        ii = torch.arange(m, device=device)
        blk[:, ii, ii] = diag[idx]
        return blk

    entries = bie_offdiag_entries(N, device)
    return _assemble(shape, leaf_fn, entries, seed, device, symmetric=False, stats=stats)


def kernel_hodlr(shape: HodlrShape, dim: int, kind: str, scale: float, nugget: float, device="cpu", seed=1,
                 stats=None):
    """HODLR operator of a symmetric kernel matrix on kd-ordered uniform points.
    kind 'gaussian': exp(-d^2 / (2 scale^2)); kind 'matern32':
    (1 + sqrt(3) d / scale) exp(-sqrt(3) d / scale). Returns (D, U, V, points)."""
    shape.validate()
    N, m = shape.N, shape.m
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    pts = torch.rand(N, dim, generator=g, device=device, dtype=torch.float64)
    pts = pts[kd_order(pts, m)].contiguous()
    p32 = pts.float()

    def kfun(d2):
        if kind == "gaussian":
            return torch.exp(-d2 / (2 * scale * scale))
        d = torch.sqrt(torch.clamp(d2, min=0))
        a = math.sqrt(3) * d / scale
        return (1 + a) * torch.exp(-a)

    def leaf_fn(b0, b1):
        P = pts[b0 * m:b1 * m].view(b1 - b0, m, dim)
        d2 = ((P[:, :, None, :] - P[:, None, :, :]) ** 2).sum(-1)
        K = kfun(d2)
        ii = torch.arange(m, device=device)
        K[:, ii, ii] += nugget
        return K

    def entries(rows, cols):
        d2 = ((p32[rows][:, :, None, :] - p32[cols][:, None, :, :]) ** 2).sum(-1)
        return kfun(d2)

    D, U, V = _assemble(shape, leaf_fn, entries, seed, device, symmetric=True, stats=stats)
    return D, U, V, pts
