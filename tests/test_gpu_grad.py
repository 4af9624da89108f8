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


@pytest.mark.parametrize("N,L,r,k", [(256, 2, 4, 1), (384, 3, 5, 2), (512, 3, 8, 3), (1024, 4, 16, 2),
                                     (2048, 3, 32, 1), (512, 1, 7, 2)])
def test_grad_matches_dense_oracle(cuda_lib, N, L, r, k):
    hb = cuda_lib
    (Dm, Um, Vm, Bm), (D, U, V, B) = make(N, L, r, k, seed=N + r)
    F = hb.hodlr_factor(D, U, V, L, r, "fp64")
    loss, dD, dU, dV, dB = hb.hodlr_grad(F, U, V, B)
    gD, gU, gV, gB = dense_grad(Dm, Um, Vm, L, Bm)
    assert loss == pytest.approx(dense_loss(Dm, Um, Vm, L, Bm), rel=1e-11)
    assert rel(dB.cpu().numpy(), gB) < 1e-10
    assert rel(dD.cpu().numpy(), gD) < 1e-10
    assert rel(dU.cpu().numpy(), gU) < 1e-10
    assert rel(dV.cpu().numpy(), gV) < 1e-10


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
    assert rel(D.grad.cpu().numpy(), 2 * gD) < 1e-10
    assert rel(U.grad.cpu().numpy(), 2 * gU) < 1e-10
    assert rel(V.grad.cpu().numpy(), 2 * gV) < 1e-10
    assert rel(B.grad.cpu().numpy(), 2 * gB) < 1e-10
