"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances. The FP64 path and the oracle are both backward-stable
eliminations of the same operator (LU with partial pivoting at the leaves;
the GPU inverts each 2r x 2r coupling matrix by Gauss-Jordan where the oracle
calls getrf/getrs), so their solutions differ by about cond(A) * u with
u = 2^-53; the synthetic operators here have cond(A) < 1e2, hence the bound
1e-11 on the relative solution difference (1e3 margin) and on the log-det
difference relative to max(1, |log det|). Refined mixed-precision solves must
reach the target residual 1e-10, measured with the oracle's own matvec.
"""
import numpy as np
import pytest
import torch

from oracle.hodlr import RecursiveHODLR, assemble_dense, matvec as o_matvec
from synth import HodlrShape, gaussian_rhs, synthetic_hodlr, to_math

pytestmark = pytest.mark.gpu

SOL_TOL = 1e-11
LD_TOL = 1e-11


def make_case(N, L, r, seed, shift=4.0, k=3):
    D, U, V, g = synthetic_hodlr(HodlrShape(N, L, r), shift, seed)
    B = gaussian_rhs(N, k, g)
    host = to_math(D, U, V, B)
    dev = tuple(t.to("cuda") for t in (D, U, V, B))
    return host, dev


def relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def close(got, ref, tol, elem_tol=None):
    """Norm-wise and element-wise agreement: ||got - ref|| <= tol ||ref|| and
    |got_i - ref_i| <= elem_tol max|ref| for every element (elem_tol = tol
    unless given; a few wrong rows or one wrong leaf cannot hide under the
    norm)."""
    got, ref = np.asarray(got), np.asarray(ref)
    assert got.shape == ref.shape
    assert relerr(got, ref) < tol
    et = tol if elem_tol is None else elem_tol
    np.testing.assert_allclose(got, ref, rtol=0, atol=et * max(np.abs(ref).max(), 1e-300))


def relres_oracle(Dm, Um, Vm, L, B, X):
    R = B - o_matvec(Dm, Um, Vm, L, X)
    return max(np.linalg.norm(R[:, j]) / np.linalg.norm(B[:, j]) for j in range(B.shape[1]))


# (N, L, r): m = N >> L
SHAPES = [
    (256, 2, 4),        # m 64
    (384, 3, 5),        # m 48, odd rank: partial warps and tiles
    (200, 3, 1),        # m 25, rank 1
    (128, 1, 3),        # one level
    (4096, 6, 16),      # the N = 4096 synthetic configuration
    (2048, 3, 32),      # m 256: leaf LU outside shared memory
    (1024, 4, 64),      # maximum rank
    (1 << 14, 6, 8),    # top levels split into several row chunks per node
]


@pytest.mark.parametrize("N,L,r", SHAPES)
def test_fp64_factor_solve_logdet_adjoint(cuda_lib, N, L, r):
    hb = cuda_lib
    (Dm, Um, Vm, Bm), (D, U, V, B) = make_case(N, L, r, seed=N + 7 * L + r)
    rec = RecursiveHODLR(Dm, Um, Vm, L)
    F = hb.hodlr_factor(D, U, V, L, r, "fp64")
    assert hb.hodlr_factor_status(F)[0] == 0
    X = hb.hodlr_solve(F, B.clone())
    x_or = rec.solve(Bm)
    close(X.cpu().numpy(), x_or, SOL_TOL)
    Xt = hb.hodlr_solve_adjoint(F, B.clone())
    close(Xt.cpu().numpy(), rec.solve_adjoint(Bm), SOL_TOL)
    s, la = hb.hodlr_logdet(F)
    so, lao = rec.slogdet()
    assert s == so
    assert abs(la - lao) <= LD_TOL * max(1.0, abs(lao))


@pytest.mark.parametrize("N,L,r", SHAPES[:6])
def test_matvec_fp64(cuda_lib, N, L, r):
    hb = cuda_lib
    (Dm, Um, Vm, Bm), (D, U, V, B) = make_case(N, L, r, seed=3 * N + r)
    Y = hb.hodlr_matvec(D, U, V, L, r, B)
    ref = o_matvec(Dm, Um, Vm, L, Bm)
    close(Y.cpu().numpy(), ref, 1e-13)


def test_dense_c0_configuration(cuda_lib):
    """N = 4096, leaf 64, rank 16, shift 4, seed 0: factor, solve and slogdet
    against dense FP64 LU of the assembled matrix."""
    hb = cuda_lib
    (Dm, Um, Vm, Bm), (D, U, V, B) = make_case(4096, 6, 16, seed=0, k=1)
    A = assemble_dense(Dm, Um, Vm, 6)
    F = hb.hodlr_factor(D, U, V, 6, 16, "fp64")
    X = hb.hodlr_solve(F, B.clone()).cpu().numpy()
    close(X, np.linalg.solve(A, Bm), SOL_TOL)
    assert np.linalg.norm(Bm - A @ X) / np.linalg.norm(Bm) < 1e-13
    s, la = hb.hodlr_logdet(F)
    sd, lad = np.linalg.slogdet(A)
    assert s == sd and abs(la - lad) <= LD_TOL * abs(lad)


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16"])
@pytest.mark.parametrize("N,L,r", [(256, 2, 4), (384, 3, 5), (800, 3, 8), (4096, 6, 16), (2048, 3, 32),
                                   (1024, 4, 64), (1 << 14, 6, 8), (1 << 13, 6, 16), (1 << 14, 7, 32)])
def test_mixed_refined_reaches_1e10(cuda_lib, prec, N, L, r):
    hb = cuda_lib
    (Dm, Um, Vm, Bm), (D, U, V, B) = make_case(N, L, r, seed=11 * N + r, k=2)
    F = hb.hodlr_factor(D, U, V, L, r, prec)
    X, it, rr, code = hb.hodlr_solve_refined(F, D, U, V, B, tol=1e-10, max_iter=60)
    Xh = X.cpu().numpy()
    assert rr <= 1e-10
    assert relres_oracle(Dm, Um, Vm, L, Bm, Xh) <= 2e-10
    close(Xh, RecursiveHODLR(Dm, Um, Vm, L).solve(Bm), 1e-8)
    # the low-precision factor's log-determinant, FP64-accumulated
    s, la = hb.hodlr_logdet(F)
    so, lao = RecursiveHODLR(Dm, Um, Vm, L).slogdet()
    assert s == so
    # FP32 leaf pivots (D truncated to FP32) and coupling matrices from FP32 /
    # BF16 panels: the log-determinant is dominated by the leaves, whose FP32
    # pivots carry ~1e-7 relative error; the couplings of these operators are
    # near the identity, so BF16 panels add little (bounds 1e-5 / 1e-4 leave
    # orders of margin over the measured errors)
    assert abs(la - lao) <= (1e-5 if prec == "fp32" else 1e-4) * max(1.0, abs(lao))


@pytest.mark.parametrize("N,L,r", [(1 << 14, 7, 32), (1 << 15, 7, 64), (1 << 16, 9, 32)])
def test_tf32_factor_projects_on_tensor_cores(cuda_lib, N, L, r):
    """The TF32 factor (FP32 panels, projections on tcgen05 kind::tf32) runs
    every level's projection on the tensor cores and agrees with the FP32
    factor to TF32 rounding (operands with a 10-bit significand: products
    within 2^-11 relative, FP32 accumulation): solutions within 1e-2 of each
    other and of the oracle's exact solve, refined to the target residual (1e-10)."""
    hb = cuda_lib
    (Dm, Um, Vm, Bm), (D, U, V, B) = make_case(N, L, r, seed=91 + r, k=2)
    F32 = hb.hodlr_factor(D, U, V, L, r, "fp32")
    X32 = hb.hodlr_solve(F32, B.clone()).cpu().numpy()
    hb.hodlr_profile_reset()
    hb.hodlr_profile_enable(True)
    Ft = hb.hodlr_factor(D, U, V, L, r, "tf32")
    hb.hodlr_profile_enable(False)
    assert hb.hodlr_profile_read()["project_tc"][1] == L
    assert hb.hodlr_factor_status(Ft)[0] == 0
    Xt = hb.hodlr_solve(Ft, B.clone()).cpu().numpy()
    close(Xt, X32, 1e-2)
    close(Xt, RecursiveHODLR(Dm, Um, Vm, L).solve(Bm), 1e-2)
    X, it, rr, code = hb.hodlr_solve_refined(Ft, D, U, V, B, tol=1e-10, max_iter=60)
    assert code == 0 and rr <= 1e-10


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_gmres_reaches_1e10(cuda_lib, prec):
    hb = cuda_lib
    N, L, r = 4096, 5, 16
    (Dm, Um, Vm, Bm), (D, U, V, B) = make_case(N, L, r, seed=99, k=1)
    F = hb.hodlr_factor(D, U, V, L, r, prec)
    X, it, rr, code = hb.hodlr_gmres(F, D, U, V, B, tol=1e-10, restart=30, max_iter=300)
    assert rr <= 1e-10
    assert relres_oracle(Dm, Um, Vm, L, Bm, X.cpu().numpy()) <= 2e-10


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("N,L,r", [(256, 1, 3), (1 << 12, 5, 7), (1 << 14, 7, 32), (1 << 15, 8, 16),
                                   (1 << 16, 9, 32)])
def test_one_column_solve_matches_multi_column(cuda_lib, prec, N, L, r):
    """The one-column preconditioner solve (two launches per level: parent
    sums + coupling solve, update fused with the next projection; leaves of
    128 rows, node sizes 128 .. N/2 so parts of one warp up to many CTAs per
    node) against the general k-column path on the same factor (column 0 of
    a two-column solve of [b, b]) -- the same FP32 arithmetic in another
    summation order -- and against the oracle's exact solve at the factor's
    precision."""
    hb = cuda_lib
    (Dm, Um, Vm, Bm), (D, U, V, B) = make_case(N, L, r, seed=13 * N + r, k=1)
    F = hb.hodlr_factor(D, U, V, L, r, prec)
    x1 = hb.hodlr_solve(F, B.clone()).cpu().numpy()
    x2 = hb.hodlr_solve(F, torch.stack([B[:, 0], B[:, 0]]).T).cpu().numpy()  # column-major N x 2
    close(x1[:, 0], x2[:, 0], 1e-5)
    close(x1[:, 0], x2[:, 1], 1e-5)
    tol = 1e-4 if prec == "fp32" else 5e-2
    close(x1, RecursiveHODLR(Dm, Um, Vm, L).solve(Bm), tol)


def test_mixed_solve_adjoint_close_to_oracle(cuda_lib):
    hb = cuda_lib
    N, L, r = 2048, 4, 8
    (Dm, Um, Vm, Bm), (D, U, V, B) = make_case(N, L, r, seed=5)
    rec = RecursiveHODLR(Dm, Um, Vm, L)
    for prec, tol in (("fp32", 1e-4), ("bf16", 5e-2)):
        F = hb.hodlr_factor(D, U, V, L, r, prec)
        close(hb.hodlr_solve(F, B.clone()).cpu().numpy(), rec.solve(Bm), tol)
        close(hb.hodlr_solve_adjoint(F, B.clone()).cpu().numpy(), rec.solve_adjoint(Bm), tol)


# ------------------------------------------------------------- device status
def test_singular_leaf_reported(cuda_lib):
    hb = cuda_lib
    (_, _, _, _), (D, U, V, B) = make_case(512, 3, 4, seed=1)
    D[5].zero_()
    F = hb.hodlr_factor(D, U, V, 3, 4, "fp64")
    code, where, detail = hb.hodlr_factor_status(F)
    assert code == hb.HODLR_ERR_SINGULAR_LEAF and where == 5 and detail == 0


def test_nonfinite_reported(cuda_lib):
    hb = cuda_lib
    (_, _, _, _), (D, U, V, B) = make_case(512, 3, 4, seed=1)
    D[2, 3, 4] = float("nan")
    F = hb.hodlr_factor(D, U, V, 3, 4, "fp32")
    code, where, _ = hb.hodlr_factor_status(F)
    assert code == hb.HODLR_ERR_NONFINITE and where == 2


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_singular_coupling_reported(cuda_lib, prec):
    """D = I, only the level-1 bases nonzero with U_a = V_a = e_1 (alpha) and
    U_b = V_b = e_1 (beta): rows 1 and N/2+1 of A coincide and the root's
    K~ = [[1, 1], [1, 1]] has an exact zero second pivot (exact in every
    precision: the projections are exactly 1)."""
    hb = cuda_lib
    N, L, r = 256, 2, 1
    m = N >> L
    D = torch.eye(m, dtype=torch.float64).repeat(1 << L, 1, 1).transpose(1, 2).contiguous().transpose(1, 2)
    U = torch.zeros(r * L, N, dtype=torch.float64).T
    U[0, 0] = 1.0
    U[N // 2, 0] = 1.0
    V = U.clone().T.contiguous().T
    D, U, V = (t.to("cuda") for t in (D, U, V))
    F = hb.hodlr_factor(D, U, V, L, r, prec)
    code, where, detail = hb.hodlr_factor_status(F)
    assert code == hb.HODLR_ERR_SINGULAR_COUPLING and where == 1 and detail == 1
    with pytest.raises(hb.HodlrError):
        hb.hodlr_logdet(F)


@pytest.mark.parametrize("N,L,r", [(1 << 14, 7, 32), (1 << 15, 7, 64), (1 << 13, 5, 32)])
def test_bf16_tensor_core_factor_matches_cuda_core(cuda_lib, N, L, r):
    """The tcgen05/TMA panel kernels and the CUDA-core kernels compute the same
    BF16-input, FP32-accumulated products (only the summation order differs),
    so the two BF16 factors' solves agree far below BF16 rounding."""
    hb = cuda_lib
    (Dm, Um, Vm, Bm), (D, U, V, B) = make_case(N, L, r, seed=77 + r, k=2)
    try:
        hb.hodlr_tc_enable(False)
        Fc = hb.hodlr_factor(D, U, V, L, r, "bf16")
        Xc = hb.hodlr_solve(Fc, B.clone()).cpu().numpy()
        lc = hb.hodlr_logdet(Fc)
    finally:
        hb.hodlr_tc_enable(True)
    hb.hodlr_profile_reset()
    hb.hodlr_profile_enable(True)
    Ft = hb.hodlr_factor(D, U, V, L, r, "bf16")
    hb.hodlr_profile_enable(False)
    assert hb.hodlr_profile_read()["project_tc"][1] == L   # every level ran on the tensor cores
    assert hb.hodlr_factor_status(Ft)[0] == 0
    Xt = hb.hodlr_solve(Ft, B.clone()).cpu().numpy()
    lt = hb.hodlr_logdet(Ft)
    # the two factors round the same FP32 sums to BF16 (Y, V copies, Z); a
    # different summation order flips the rounding of a few entries by one
    # BF16 unit (2^-8 relative), which moves single solution entries by up to
    # the BF16 unit roundoff 2^-9 of max|x| while the norm stays near 1e-5
    close(Xt, Xc, 1e-4, elem_tol=2.0 ** -9)
    assert lt[0] == lc[0] and abs(lt[1] - lc[1]) < 1e-6 * max(1.0, abs(lc[1]))
    # and the BF16 factor is a BF16-accurate inverse of the FP64 operator
    close(Xt, RecursiveHODLR(Dm, Um, Vm, L).solve(Bm), 5e-2)


@pytest.mark.parametrize("N,L,r", [(256, 2, 4), (384, 3, 5), (128, 1, 3), (4096, 6, 16), (2048, 3, 32),
                                   (1 << 14, 6, 64), (256, 1, 4), (1 << 10, 3, 8), (1 << 12, 5, 16),
                                   (1 << 14, 7, 32), (3 << 10, 5, 24)])
def test_matvec_fp64_single_rhs(cuda_lib, N, L, r):
    """k = 1 takes the four-launch path (all levels' projections per leaf);
    leaves of 128 rows use the vectorized projection kernels (16 rows per
    lane when the leaves come in fours, 4 rows per lane otherwise)."""
    hb = cuda_lib
    (Dm, Um, Vm, Bm), (D, U, V, B) = make_case(N, L, r, seed=5 * N + r, k=1)
    Y = hb.hodlr_matvec(D, U, V, L, r, B)
    ref = o_matvec(Dm, Um, Vm, L, Bm)
    close(Y.cpu().numpy(), ref, 1e-13)


@pytest.mark.parametrize("N,L,r", [(1 << 14, 7, 32), (100 << 6, 6, 8), (1 << 13, 6, 16), (3 << 13, 8, 5)])
def test_tensor_core_leaf_inverse_matches_cuda_core(cuda_lib, N, L, r):
    """Leaves of 65..128 rows: the blocked Gauss-Jordan inverse with its
    trailing updates on the tensor cores (split TF32 operands, FP32
    accumulation) against the register Gauss-Jordan kernel on the CUDA cores.
    In the FP32 factor the switch changes only the leaf inverse, so the two
    factors differ by FP32-level rounding: solutions within 1e-5, the
    log-determinants (same pivots) within 1e-6 relative; both within the FP32
    factor's bound of the oracle's exact solve."""
    hb = cuda_lib
    (Dm, Um, Vm, Bm), (D, U, V, B) = make_case(N, L, r, seed=41 * L + r, k=2)
    try:
        hb.hodlr_tc_enable(False)
        Fc = hb.hodlr_factor(D, U, V, L, r, "fp32")
        Xc = hb.hodlr_solve(Fc, B.clone()).cpu().numpy()
        lc = hb.hodlr_logdet(Fc)
    finally:
        hb.hodlr_tc_enable(True)
    Ft = hb.hodlr_factor(D, U, V, L, r, "fp32")
    assert hb.hodlr_factor_status(Ft)[0] == 0
    Xt = hb.hodlr_solve(Ft, B.clone()).cpu().numpy()
    lt = hb.hodlr_logdet(Ft)
    close(Xt, Xc, 1e-5)
    assert lt[0] == lc[0] and abs(lt[1] - lc[1]) <= 1e-6 * max(1.0, abs(lc[1]))
    rec = RecursiveHODLR(Dm, Um, Vm, L)
    close(Xt, rec.solve(Bm), 1e-4)
    so, lao = rec.slogdet()
    assert lt[0] == so and abs(lt[1] - lao) <= 1e-5 * max(1.0, abs(lao))


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_tensor_core_leaf_inverse_reports_singular_and_nonfinite(cuda_lib, prec):
    hb = cuda_lib
    N, L, r = 1 << 10, 3, 8   # m = 128
    (_, _, _, _), (D, U, V, B) = make_case(N, L, r, seed=2)
    D1 = D.clone()
    D1[5].zero_()
    F = hb.hodlr_factor(D1, U, V, L, r, prec)
    code, where, detail = hb.hodlr_factor_status(F)
    assert code == hb.HODLR_ERR_SINGULAR_LEAF and where == 5 and detail == 0
    D2 = D.clone()
    D2[2, 3, 4] = float("inf")
    F2 = hb.hodlr_factor(D2, U, V, L, r, prec)
    code, where, _ = hb.hodlr_factor_status(F2)
    assert code == hb.HODLR_ERR_NONFINITE and where == 2


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("k,restart", [(1, 30), (3, 30), (2, 2)])
def test_gmres_lockstep_columns_reach_1e10(cuda_lib, prec, k, restart):
    """FGMRES on k right-hand sides in lockstep (one k-column preconditioner
    solve and one k-column FP64 matvec per inner iteration); restart 2 forces
    several cycles, each continuing from r - (A Z) y. Every column reaches
    the target residual (1e-10) measured by the oracle's matvec, and agrees with
    the oracle's exact solve to cond(A) * 1e-10."""
    hb = cuda_lib
    N, L, r = 4096, 5, 16
    (Dm, Um, Vm, Bm), (D, U, V, B) = make_case(N, L, r, seed=17 + k + restart, k=k)
    F = hb.hodlr_factor(D, U, V, L, r, prec)
    X, it, rr, code = hb.hodlr_gmres(F, D, U, V, B, tol=1e-10, restart=restart, max_iter=300)
    assert code == 0 and rr <= 1e-10 and it >= 1
    Xh = X.cpu().numpy()
    assert relres_oracle(Dm, Um, Vm, L, Bm, Xh) <= 2e-10
    close(Xh, RecursiveHODLR(Dm, Um, Vm, L).solve(Bm), 1e-8)


def test_refinement_hands_over_to_fgmres(cuda_lib):
    """Refinement that stops without reaching tol (here: no corrections
    allowed) continues with FGMRES(30) from its iterate when restart > 0, and
    reports NOT_CONVERGED without it."""
    hb = cuda_lib
    N, L, r = 4096, 5, 16
    (Dm, Um, Vm, Bm), (D, U, V, B) = make_case(N, L, r, seed=23, k=2)
    F = hb.hodlr_factor(D, U, V, L, r, "bf16")
    X, it, rr, code = hb.hodlr_solve_refined(F, D, U, V, B, tol=1e-10, max_iter=0, restart=30, gmres_max_iter=300)
    assert code == 0 and rr <= 1e-10 and it >= 1
    assert relres_oracle(Dm, Um, Vm, L, Bm, X.cpu().numpy()) <= 2e-10
    X2, it2, rr2, code2 = hb.hodlr_solve_refined(F, D, U, V, B, tol=1e-10, max_iter=0, restart=0,
                                                 raise_on_fail=False)
    assert code2 == hb.HODLR_ERR_NOT_CONVERGED and it2 == 0 and rr2 > 1e-10


@pytest.mark.parametrize("N,L,r", [(4096, 6, 16), (2048, 3, 32)])
def test_inplace_fp64_factor(cuda_lib, N, L, r):
    """The in-place FP64 factor (leaf LUs over D, Y_big over U) solves,
    adjoint-solves and gives the log-determinant as the out-of-place one, to
    the oracle's tolerance, from a smaller workspace."""
    hb = cuda_lib
    (Dm, Um, Vm, Bm), (D, U, V, B) = make_case(N, L, r, seed=N + 3 * r, k=2)
    rec = RecursiveHODLR(Dm, Um, Vm, L)
    F = hb.hodlr_factor(D, U, V, L, r, "fp64")
    D2, U2 = D.clone(), U.clone()   # clone keeps the column-major strides
    assert D2.stride() == D.stride() and U2.stride() == U.stride()
    Fi = hb.hodlr_factor_inplace(D2, U2, V, L, r)
    assert hb.hodlr_factor_status(Fi)[0] == 0
    assert Fi.workspace.numel() < F.workspace.numel()
    assert not torch.equal(D2, D) and not torch.equal(U2, U)   # overwritten
    close(hb.hodlr_solve(Fi, B.clone()).cpu().numpy(), rec.solve(Bm), SOL_TOL)
    close(hb.hodlr_solve_adjoint(Fi, B.clone()).cpu().numpy(), rec.solve_adjoint(Bm), SOL_TOL)
    s, la = hb.hodlr_logdet(Fi)
    so, lao = rec.slogdet()
    assert s == so and abs(la - lao) <= LD_TOL * max(1.0, abs(lao))
