"""Full-size GPU checks at the sizes of the benchmark configurations, in the
launch configuration bench.py times (same N, leaf, rank, right-hand sides,
factor precision and outer solver), on seeded synthetic operators of those
shapes.

The oracle cannot factor these sizes in test time, so the checks are the
ones it can make one row at a time (``sampled_rows_matvec``) or properties
that hold at any size:
* the FP64 matvec agrees with the oracle's row-by-row product on sampled rows;
* the mixed-precision solve reaches the FP64 relative residual <= 1e-10, and
  the residual rows the oracle recomputes from the returned X are within that
  bound (|r_i| <= ||r||_2 <= tol ||b||_2 for every row i);
* the low-precision factor's log-determinant has the FP64 factor's sign and
  agrees with it to the low precision.
"""
import numpy as np
import pytest
import torch

from oracle.hodlr import sampled_rows_matvec
from synth import HodlrShape, gaussian_rhs, synthetic_hodlr

pytestmark = pytest.mark.gpu

# (N, L, r, k, precision, solver, leaf shift): the benchmark configurations'
# shapes (BIE 2^20 / leaf 128 / rank 32 / 1 RHS with FGMRES; Gaussian 2^18 /
# leaf 256 / rank 64 / 16 RHS; Matern 2^20 / leaf 256 / rank 64 / 32 RHS)
FULL = [
    (1 << 20, 13, 32, 1, "bf16", "gmres", 4.0),
    (1 << 18, 10, 64, 16, "fp32", "refine", 4.0),
    (1 << 20, 12, 64, 32, "fp32", "refine", 4.0),
]


def _host(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("N,L,r,k,prec,solver,shift", FULL)
def test_fullsize_solve_matvec_logdet(cuda_lib, N, L, r, k, prec, solver, shift):
    hb = cuda_lib
    D, U, V, g = synthetic_hodlr(HodlrShape(N, L, r), shift, seed=N + r, device="cuda")
    B = gaussian_rhs(N, k, g, device="cuda")
    rng = np.random.default_rng(N + k)
    rows = np.sort(rng.choice(N, size=24, replace=False))
    rows = np.unique(np.concatenate([rows, [0, N // 2 - 1, N // 2, N - 1]]))
    Dh = _host(D)
    Uh, Vh = _host(U), _host(V)

    # FP64 matvec vs the oracle, row by row
    Y = hb.hodlr_matvec(D, U, V, L, r, B)
    ref = sampled_rows_matvec(Dh, Uh, Vh, L, _host(B), rows)
    got = _host(Y)[rows]
    assert np.abs(got - ref).max() <= 1e-12 * max(np.abs(ref).max(), 1.0)

    # mixed-precision factor + the benchmark's outer solver
    F = hb.hodlr_factor(D, U, V, L, r, prec)
    if solver == "gmres":
        X, it, rr, code = hb.hodlr_gmres(F, D, U, V, B, tol=1e-10, restart=30, max_iter=300)
    else:
        X, it, rr, code = hb.hodlr_solve_refined(F, D, U, V, B, tol=1e-10, max_iter=50)
    assert code == 0 and rr <= 1e-10
    Bh, Xh = _host(B), _host(X)
    R = Bh[rows] - sampled_rows_matvec(Dh, Uh, Vh, L, Xh, rows)
    bn = np.linalg.norm(Bh, axis=0)
    assert (np.abs(R) <= 1.5e-10 * bn[None, :]).all()

    # log-determinant: the low-precision factor against the FP64 factor
    s_lo, ld_lo = hb.hodlr_logdet(F)
    del F
    torch.cuda.empty_cache()
    F64 = hb.hodlr_factor(D, U, V, L, r, "fp64")
    s64, ld64 = hb.hodlr_logdet(F64)
    assert s_lo == s64
    tol = 1e-4 if prec == "bf16" else 1e-5
    assert abs(ld_lo - ld64) <= tol * max(1.0, abs(ld64))
