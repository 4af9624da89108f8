"""The operator the benchmark times, against the oracle.

The 2D Laplace double-layer BIE on the star curve (leaf 128, rank 32, one
right-hand side; the structure of the Sec. 4.2 experiments) at N = 2^14 and
2^16, generated exactly as ``bench.py`` generates it (seed 2; right-hand side
from the generator seeded 2 + 1000 * rank). Two call sequences:

* the benchmark's: BF16 factor -> hodlr_gmres (FGMRES(30), tol 1e-10) ->
  hodlr_logdet;
* the plain FP64 one: FP64 factor -> hodlr_solve -> hodlr_logdet.

Both are compared element by element with the oracle's recursive solve and
its log-determinant (Sec. 3.1 Theorem 1, Sec. 3.5).

Tolerances. The FP64 factor and the oracle are two backward-stable
eliminations of the same operator; this second-kind operator is well
conditioned (cond(A) ~ 10), so their solutions agree to 1e-11 and the
log-determinants to 1e-11 relative. FGMRES stops at relres <= 1e-10, so its
x is within cond(A) * 1e-10 of the exact solution: 1e-8 element-wise (relative
to max|x|) leaves a margin of 10. The BF16 factor's log-determinant is an
approximation (coupling matrices formed from BF16 panels, FP32 leaf
pivots); its error against the FP64 value is reported by the benchmark and
bounded here by 1e-5 relative (measured: 9.3e-7 at N = 2^14, 3.7e-7 at
2^16).
"""
import numpy as np
import pytest
import torch

from oracle.hodlr import RecursiveHODLR, matvec as o_matvec
from synth import HodlrShape, gaussian_rhs, to_math
from synth.kernels import bie_hodlr

pytestmark = pytest.mark.gpu


def close(got, ref, tol):
    got, ref = np.asarray(got), np.asarray(ref)
    assert got.shape == ref.shape
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
    np.testing.assert_allclose(got, ref, rtol=0, atol=tol * np.abs(ref).max())


@pytest.mark.parametrize("N,L", [(1 << 14, 7), (1 << 16, 9)])
def test_bie_bench_sequence_against_oracle(cuda_lib, N, L):
    hb = cuda_lib
    r, seed = 32, 2
    D, U, V = bie_hodlr(HodlrShape(N, L, r), device="cuda", seed=seed)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    B = gaussian_rhs(N, 1, g, device="cuda")
    Dm, Um, Vm, Bm = to_math(D, U, V, B)
    rec = RecursiveHODLR(Dm, Um, Vm, L)
    x_or = rec.solve(Bm)
    s_or, ld_or = rec.slogdet()

    # the benchmark's sequence
    F = hb.hodlr_factor(D, U, V, L, r, "bf16")
    X, it, rr, code = hb.hodlr_gmres(F, D, U, V, B, tol=1e-10, restart=30, max_iter=300)
    s_lo, ld_lo = hb.hodlr_logdet(F)
    assert code == 0 and rr <= 1e-10
    Xh = X.cpu().numpy()
    res = Bm - o_matvec(Dm, Um, Vm, L, Xh)
    assert np.linalg.norm(res) <= 1.5e-10 * np.linalg.norm(Bm)
    close(Xh, x_or, 1e-8)
    assert s_lo == s_or
    ld_err = abs(ld_lo - ld_or) / abs(ld_or)
    assert ld_err <= 1e-5, ld_err

    # plain FP64
    F64 = hb.hodlr_factor(D, U, V, L, r, "fp64")
    X64 = hb.hodlr_solve(F64, B.clone()).cpu().numpy()
    close(X64, x_or, 1e-11)
    s64, ld64 = hb.hodlr_logdet(F64)
    assert s64 == s_or
    assert abs(ld64 - ld_or) <= 1e-11 * abs(ld_or)
    print(f"N={N}: FGMRES {it} iterations, relres {rr:.2e}, |x_bf16 - x_or|/|x_or| "
          f"{np.linalg.norm(Xh - x_or) / np.linalg.norm(x_or):.2e}, logdet bf16 rel err {ld_err:.2e}, "
          f"fp64 rel err {abs(ld64 - ld_or) / abs(ld_or):.2e}")
