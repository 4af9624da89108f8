"""Variable ranks (Eq. e:u with per-level / per-node ranks), GPU side.

* hodlr_pack_level_ranks: a ragged operator (level c's bases in r_c columns,
  some nodes of lower rank with zero columns at the right) packed into the
  uniform layout is the same matrix: the live columns are copied exactly, the
  padding is zero, and its FP64 factor / BF16 + refinement solves match the
  dense solve of the oracle's ragged assembly element-wise.
* hodlr_compress with a pivot tolerance: per-block ranks below the maximum,
  bases beyond each block's rank exactly zero, the assembled approximation
  close to the dense BIE matrix, and the operator solvable to 1e-10.
"""
import numpy as np
import pytest
import torch

from oracle.hodlr import assemble_dense, assemble_dense_level_ranks
from synth.kernels import bie_dense

pytestmark = pytest.mark.gpu


def test_pack_level_ranks_and_solve(cuda_lib):
    hb = cuda_lib
    N, L = 4096, 5
    m = N >> L
    ranks = [12, 10, 8, 6, 5]
    rng = np.random.default_rng(8)
    D = rng.standard_normal((1 << L, m, m)) / np.sqrt(m) + 4.0 * np.eye(m)
    cols = sum(ranks)
    Ur = np.zeros((N, cols))
    Vr = np.zeros((N, cols))
    off = 0
    for c in range(1, L + 1):
        n = N >> c
        for node in range(1 << c):
            rk = ranks[c - 1] - (node % 3)          # some nodes of lower rank: zero columns at the right
            rows = slice(node * n, (node + 1) * n)
            Ur[rows, off:off + rk] = rng.standard_normal((n, rk)) * 0.5 / np.sqrt(n)
            Vr[rows, off:off + rk] = rng.standard_normal((n, rk)) * 0.5 / np.sqrt(n)
        off += ranks[c - 1]
    A = assemble_dense_level_ranks(D, Ur, Vr, L, ranks)
    b = rng.standard_normal((N, 2))
    x = np.linalg.solve(A, b)
    dev = torch.device("cuda")
    Dd = torch.from_numpy(D.transpose(0, 2, 1).copy()).to(dev).transpose(1, 2)   # column-major blocks
    Urd = torch.from_numpy(Ur.T.copy()).to(dev).T
    Vrd = torch.from_numpy(Vr.T.copy()).to(dev).T
    Bd = torch.from_numpy(b.T.copy()).to(dev).T
    U, V = hb.hodlr_pack_level_ranks(Urd, Vrd, L, ranks)
    r = max(ranks)
    Uh, Vh = U.cpu().numpy(), V.cpu().numpy()
    off = 0
    for c in range(1, L + 1):
        rc = ranks[c - 1]
        assert np.array_equal(Uh[:, (c - 1) * r:(c - 1) * r + rc], Ur[:, off:off + rc])
        assert np.array_equal(Vh[:, (c - 1) * r:(c - 1) * r + rc], Vr[:, off:off + rc])
        assert not Uh[:, (c - 1) * r + rc:c * r].any() and not Vh[:, (c - 1) * r + rc:c * r].any()
        off += rc
    assert np.allclose(assemble_dense(D, Uh, Vh, L), A, rtol=0, atol=1e-14)
    F = hb.hodlr_factor(Dd, U, V, L, r, "fp64")
    X = hb.hodlr_solve(F, Bd.clone()).cpu().numpy()
    np.testing.assert_allclose(X, x, rtol=0, atol=1e-11 * np.abs(x).max())
    s, la = hb.hodlr_logdet(F)
    sd, lad = np.linalg.slogdet(A)
    assert s == sd and abs(la - lad) <= 1e-11 * abs(lad)
    Fb = hb.hodlr_factor(Dd, U, V, L, r, "bf16")
    Xb, it, rr, code = hb.hodlr_solve_refined(Fb, Dd, U, V, Bd, tol=1e-10, max_iter=50)
    assert code == 0 and rr <= 1e-10
    np.testing.assert_allclose(Xb.cpu().numpy(), x, rtol=0, atol=1e-8 * np.abs(x).max())


def test_compress_with_tolerance_gives_variable_ranks(cuda_lib):
    hb = cuda_lib
    N, L, r = 4096, 5, 32
    D, U, V, ranks = hb.hodlr_compress(N, L, r, "bie_star", tol=1e-6, want_ranks=True)
    rk = ranks.cpu().numpy()
    Uh, Vh = U.cpu().numpy(), V.cpu().numpy()
    assert rk.max() <= r and rk.min() >= 1 and rk.min() < r   # tolerance-driven: below the cap
    for c in range(1, L + 1):
        n = N >> c
        for blk in range(1 << c):
            k = int(rk[(1 << c) - 2 + blk])
            cols = slice((c - 1) * r + k, c * r)
            assert not Uh[blk * n:(blk + 1) * n, cols].any()          # u's of the block beyond its rank
            assert not Vh[(blk ^ 1) * n:((blk ^ 1) + 1) * n, cols].any()
    A = bie_dense(N).numpy()
    err = np.linalg.norm(assemble_dense(D.cpu().numpy(), Uh, Vh, L) - A) / np.linalg.norm(A)
    print(f"bie_star tol 1e-6: ranks {int(rk.min())}..{int(rk.max())}, |A_hodlr - A|_F / |A|_F = {err:.2e}")
    assert err <= 1e-5
    g = torch.Generator(device="cuda").manual_seed(3)
    B = torch.randn(1, N, generator=g, device="cuda", dtype=torch.float64).T
    F = hb.hodlr_factor(D, U, V, L, r, "bf16")
    X, it, rr, code = hb.hodlr_gmres(F, D, U, V, B, tol=1e-10, restart=30, max_iter=300)
    assert code == 0 and rr <= 1e-10
