"""Checks of the seeded input generators (CPU): the boundary-integral matrix
satisfies Gauss's identity, kd-tree orders are valid permutations with
median splits, compression keeps leaf blocks exact and the off-diagonal
error small, and symmetric kernels give U = V."""
import numpy as np
import pytest
import torch

from oracle.hodlr import assemble_dense
from synth import HodlrShape, to_math
from synth.kernels import bie_dense, bie_hodlr, kd_order, kernel_hodlr, star_curve


@pytest.mark.parametrize("N", [256, 1024])
def test_bie_gauss_identity(N):
    """The double layer potential of a constant density is -1/2 on the curve
    (outward normal), so (-1/2 I + D) 1 = -1 up to the trapezoid rule's
    (spectral) error."""
    A = bie_dense(N)
    err = (A @ torch.ones(N, dtype=torch.float64) + 1).abs().max().item()
    assert err < 1e-12


def test_star_curve_geometry():
    x, n, w, kappa = star_curve(4096)
    assert torch.allclose(n.norm(dim=1), torch.ones(4096, dtype=torch.float64))
    # perimeter and enclosed area (shoelace) of rho = 1 + 0.3 cos 5t
    area = 0.5 * (x[:, 0] * torch.roll(x[:, 1], -1) - torch.roll(x[:, 0], -1) * x[:, 1]).sum().item()
    assert area == pytest.approx(np.pi * (1 + 0.3 ** 2 / 2), rel=1e-5)  # polygon error O(N^-2)
    # total turning of a simple closed curve: integral of curvature = 2 pi
    assert (kappa * w).sum().item() == pytest.approx(2 * np.pi, rel=1e-10)


def test_bie_hodlr_compression():
    s = HodlrShape(1024, 3, 16)
    D, U, V = bie_hodlr(s)
    Dm, Um, Vm = to_math(D, U, V)
    A = bie_dense(1024).numpy()
    Ah = assemble_dense(Dm, Um, Vm, 3)
    for b in range(8):
        sl = slice(b * 128, (b + 1) * 128)
        np.testing.assert_allclose(Ah[sl, sl], A[sl, sl], rtol=0, atol=1e-15)
    assert np.linalg.norm(Ah - A) / np.linalg.norm(A) < 1e-4


def test_kd_order():
    g = torch.Generator().manual_seed(0)
    pts = torch.rand(256, 2, generator=g, dtype=torch.float64)
    perm = kd_order(pts, 16)
    assert sorted(perm.tolist()) == list(range(256))
    P = pts[perm]
    # first split on x at the median, second on y within each half
    assert P[:128, 0].max() <= P[128:, 0].min()
    assert P[:64, 1].max() <= P[64:128, 1].min()
    assert P[128:192, 1].max() <= P[192:, 1].min()


@pytest.mark.parametrize("dim,kind,scale,nugget", [(2, "gaussian", 0.1, 1e-2), (3, "matern32", 0.2, 1e-3)])
def test_kernel_hodlr_symmetric(dim, kind, scale, nugget):
    s = HodlrShape(1024, 2, 32)
    D, U, V, pts = kernel_hodlr(s, dim, kind, scale, nugget)
    assert torch.equal(U, V)
    Dm, Um, Vm = to_math(D, U, V)
    Ah = assemble_dense(Dm, Um, Vm, 2)
    np.testing.assert_allclose(Ah, Ah.T, atol=1e-15)
    d = torch.cdist(pts, pts)
    if kind == "gaussian":
        K = torch.exp(-d ** 2 / (2 * scale ** 2))
    else:
        a = np.sqrt(3) * d / scale
        K = (1 + a) * torch.exp(-a)
    K = K + nugget * torch.eye(1024, dtype=torch.float64)
    for b in range(4):
        sl = slice(b * 256, (b + 1) * 256)
        np.testing.assert_allclose(Ah[sl, sl], K.numpy()[sl, sl], rtol=0, atol=1e-12)
    # fixed rank 32 on 512-point blocks: a few percent in 3D, far less in 2D
    assert np.linalg.norm(Ah - K.numpy()) / np.linalg.norm(K.numpy()) < (5e-3 if dim == 2 else 5e-2)


@pytest.mark.parametrize("N", [1 << 14, 1 << 16])
def test_bie_offdiag_entries_match_fp64(N):
    """The generator's mixed-precision entries (FP64 within the band, FP64
    differences elsewhere, FP32 rest) against the FP64 formula on sibling
    blocks of several levels, both ends of each block (the periodic wrap
    included): within 2e-6 of the block's largest entry (FP32 output rounding
    alone is 6e-8 of an entry; coordinates in FP32 would give 1e-2 and more)."""
    from synth.kernels import bie_block, bie_offdiag_entries
    x, nrm, w, _ = star_curve(N)
    ent = bie_offdiag_entries(N)
    for c in (1, 2, 4, 6):
        n = N >> c
        for blk in (0, 1, (1 << c) - 1):
            cols = torch.arange((blk ^ 1) * n, ((blk ^ 1) + 1) * n)
            for lo in (blk * n, blk * n + n - min(n, 256)):
                rows = torch.arange(lo, lo + min(n, 256))
                got = ent(rows[None, :], cols[None, :])[0].double()
                ref = bie_block(x, nrm, w, rows[None, :], cols[None, :])[0]
                assert ((got - ref).abs().max() / ref.abs().max()).item() <= 2e-6, (N, c, blk, lo)
