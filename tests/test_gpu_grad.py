"""Gradients of sum_j b_j^T A^{-1} b_j + log|det A| (FP64 factor, hodlr_grad)
against the oracle's dense gradient (matrix calculus on the assembled A,
itself pinned by finite differences and torch autograd in test_oracle.py) and
against central finite differences of the GPU loss along random directions
(relative 1e-6)."""
import numpy as np
import pytest
import torch

from oracle.hodlr import dense_grad, dense_loss
from synth import HodlrShape, gaussian_rhs, synthetic_hodlr, to_math

pytestmark = pytest.mark.gpu


def make(N, L, r, k, seed):
    D, U, V, g = synthetic_hodlr(HodlrShape(N, L, r), 4.0, seed)
    B = gaussian_rhs(N, k, g)
    return to_math(D, U, V, B), tuple(t.to("cuda") for t in (D, U, V, B))


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def close(got, ref, tol):
    """Norm-wise and element-wise: every entry within tol * max|ref|."""
    got, ref = np.asarray(got), np.asarray(ref)
    assert got.shape == ref.shape
    assert rel(got, ref) < tol
    np.testing.assert_allclose(got, ref, rtol=0, atol=tol * max(np.abs(ref).max(), 1e-300))


@pytest.mark.parametrize("N,L,r,k", [(256, 2, 4, 1), (384, 3, 5, 2), (512, 3, 8, 3), (1024, 4, 16, 2),
                                     (2048, 3, 32, 1), (512, 1, 7, 2)])
def test_grad_matches_dense_oracle(cuda_lib, N, L, r, k):
    hb = cuda_lib
    (Dm, Um, Vm, Bm), (D, U, V, B) = make(N, L, r, k, seed=N + r)
    F = hb.hodlr_factor(D, U, V, L, r, "fp64")
    loss, dD, dU, dV, dB = hb.hodlr_grad(F, U, V, B)
    gD, gU, gV, gB = dense_grad(Dm, Um, Vm, L, Bm)
    assert loss == pytest.approx(dense_loss(Dm, Um, Vm, L, Bm), rel=1e-11)
    close(dB.cpu().numpy(), gB, 1e-10)
    close(dD.cpu().numpy(), gD, 1e-10)
    close(dU.cpu().numpy(), gU, 1e-10)
    close(dV.cpu().numpy(), gV, 1e-10)


def test_grad_finite_differences(cuda_lib):
    hb = cuda_lib
    N, L, r, k = 1024, 4, 8, 2
    (_, _, _, _), (D, U, V, B) = make(N, L, r, k, seed=3)
    F = hb.hodlr_factor(D, U, V, L, r, "fp64")
    loss, dD, dU, dV, dB = hb.hodlr_grad(F, U, V, B)
    g = torch.Generator(device="cuda").manual_seed(11)

    def loss_at(Dp, Up, Vp, Bp):
        Fp = hb.hodlr_factor(Dp, Up, Vp, L, r, "fp64")
        return hb.hodlr_grad(Fp, Up, Vp, Bp)[0]

    for _ in range(5):
        dirs = [torch.randn(t.shape, generator=g, device="cuda", dtype=torch.float64) for t in (D, U, V, B)]
        # keep the layouts of the inputs
        dirs = [dd.transpose(1, 2).contiguous().transpose(1, 2) if i == 0 else dd.T.contiguous().T
                for i, dd in enumerate(dirs)]
        h = 1e-6
        plus = [t + h * dd for t, dd in zip((D, U, V, B), dirs)]
        minus = [t - h * dd for t, dd in zip((D, U, V, B), dirs)]
        plus = [p.transpose(1, 2).contiguous().transpose(1, 2) if i == 0 else p.T.contiguous().T
                for i, p in enumerate(plus)]
        minus = [p.transpose(1, 2).contiguous().transpose(1, 2) if i == 0 else p.T.contiguous().T
                 for i, p in enumerate(minus)]
        fd = (loss_at(*plus) - loss_at(*minus)) / (2 * h)
        an = sum(float((gr * dd).sum()) for gr, dd in zip((dD, dU, dV, dB), dirs))
        assert fd == pytest.approx(an, rel=1e-6)


def test_autograd_function(cuda_lib):
    from paper_2208_06290_gb300.autograd import hodlr_solve_logdet
    N, L, r, k = 512, 3, 4, 2
    (Dm, Um, Vm, Bm), (D, U, V, B) = make(N, L, r, k, seed=21)
    for t in (D, U, V, B):
        t.requires_grad_(True)
    loss = hodlr_solve_logdet(D, U, V, B, L, r)
    (2.0 * loss).backward()
    gD, gU, gV, gB = dense_grad(Dm, Um, Vm, L, Bm)
    close(D.grad.cpu().numpy(), 2 * gD, 1e-10)
    close(U.grad.cpu().numpy(), 2 * gU, 1e-10)
    close(V.grad.cpu().numpy(), 2 * gV, 1e-10)
    close(B.grad.cpu().numpy(), 2 * gB, 1e-10)


@pytest.mark.parametrize("N,L,r,k", [(1024, 3, 16, 2), (2048, 4, 32, 1), (4096, 4, 64, 3)])
def test_grad_fp32_factor_against_dense_fp64(cuda_lib, N, L, r, k):
    """The gradient computed with an FP32 factor (FP32 solves, Y_big and leaf
    inverses; FP64 coupling inverses, log-dets and accumulations) against the
    dense FP64 gradient: its error is the FP32 factor's solve accuracy carried
    into the blocks, about 1e-6 for these operators (cond(A) < 1e2); bounded
    by 1e-4 norm-wise and element-wise (relative to the block's max)."""
    hb = cuda_lib
    (Dm, Um, Vm, Bm), (D, U, V, B) = make(N, L, r, k, seed=5 * N + r)
    F = hb.hodlr_factor(D, U, V, L, r, "fp32")
    loss, dD, dU, dV, dB = hb.hodlr_grad(F, U, V, B)
    gD, gU, gV, gB = dense_grad(Dm, Um, Vm, L, Bm)
    assert loss == pytest.approx(dense_loss(Dm, Um, Vm, L, Bm), rel=1e-5)
    errs = {}
    for name, got, ref in (("dB", dB, gB), ("dD", dD, gD), ("dU", dU, gU), ("dV", dV, gV)):
        got = got.cpu().numpy()
        close(got, ref, 1e-4)
        errs[name] = rel(got, ref)
    print(f"fp32-factor gradient, N={N} r={r} k={k}: relative errors vs FP64 " +
          ", ".join(f"{n} {e:.1e}" for n, e in errs.items()))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_autograd_forward_is_loss_only_and_backward_lazy(cuda_lib, prec):
    """forward runs factor + solve + logdet only (no gradient kernels); the
    adjoint gradient runs in backward, on the forward's factor."""
    from paper_2208_06290_gb300.autograd import hodlr_solve_logdet
    hb = cuda_lib
    N, L, r, k = 1024, 3, 8, 2
    (Dm, Um, Vm, Bm), (D, U, V, B) = make(N, L, r, k, seed=31)
    for t in (D, U, V, B):
        t.requires_grad_(True)
    hb.hodlr_profile_reset()
    hb.hodlr_profile_enable(True)
    loss = hodlr_solve_logdet(D, U, V, B, L, r, prec)
    fwd = hb.hodlr_profile_read()
    loss.backward()
    hb.hodlr_profile_enable(False)
    both = hb.hodlr_profile_read()
    assert fwd["leaf_matvec"][1] == 0          # the gradient's leaf products have not run
    assert both["leaf_matvec"][1] > 0
    tol = 1e-10 if prec == "fp64" else 1e-4
    assert float(loss) == pytest.approx(dense_loss(Dm, Um, Vm, L, Bm), rel=1e-11 if prec == "fp64" else 1e-5)
    gD, gU, gV, gB = dense_grad(Dm, Um, Vm, L, Bm)
    close(D.grad.cpu().numpy(), gD, tol)
    close(U.grad.cpu().numpy(), gU, tol)
    close(V.grad.cpu().numpy(), gV, tol)
    close(B.grad.cpu().numpy(), gB, tol)
