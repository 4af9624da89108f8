"""Pins of the oracle's partial-pivoted cross approximation (construction,
Sec. 2.2) against textbook facts about it (CPU only):
* a matrix of rank s <= r is reproduced exactly (to rounding) after s steps;
* the approximation interpolates M on every pivot row and pivot column
  (the residual is zero on the cross);
* one step on a rank-1 matrix x y^T with the largest entry of its first row
  at column j gives u = M(:, j) and v = M(0, :) / M(0, j) (by hand);
* on M^T with the pivot roles exchanged it returns the transposed factors
  (the symmetric-kernel relation U_beta = V, V_alpha = U used by the GPU
  construction).
"""
import numpy as np

from oracle.hodlr import cross_approximation


def test_exact_on_low_rank():
    rng = np.random.default_rng(1)
    for s in (1, 3, 7):
        M = rng.standard_normal((60, s)) @ rng.standard_normal((s, 45))
        U, V, pr, pc = cross_approximation(M, s)
        assert np.abs(U @ V.T - M).max() <= 1e-12 * np.abs(M).max()
        assert len(pr) == s and len(pc) == s


def test_interpolates_on_the_cross():
    rng = np.random.default_rng(2)
    x = np.linspace(0, 1, 70)
    y = np.linspace(2, 3, 50)
    M = 1.0 / (x[:, None] + y[None, :]) + 1e-3 * rng.standard_normal((70, 50))
    U, V, pr, pc = cross_approximation(M, 6)
    A = U @ V.T
    for i in pr:
        assert np.allclose(A[i, :], M[i, :], rtol=0, atol=1e-12 * np.abs(M).max())
    for j in pc:
        assert np.allclose(A[:, j], M[:, j], rtol=0, atol=1e-12 * np.abs(M).max())


def test_rank_one_by_hand():
    x = np.array([1.0, -2.0, 0.5, 3.0])
    y = np.array([0.25, -4.0, 1.0])
    M = np.outer(x, y)
    U, V, pr, pc = cross_approximation(M, 1)
    assert pr == [0] and pc == [1]            # |M(0, :)| = (0.25, 4, 1): column 1
    assert np.array_equal(U[:, 0], M[:, 1])
    assert np.array_equal(V[:, 0], M[0, :] / M[0, 1])


def test_transpose_relation():
    rng = np.random.default_rng(3)
    M = rng.standard_normal((30, 30))
    U, V, pr, pc = cross_approximation(M, 5)
    # the cross of M^T taking M's pivot columns as rows and rows as columns
    # reproduces the same approximation, transposed
    Ut, Vt, _, _ = cross_approximation(M.T, 5, rows=pc, cols=pr)
    assert np.allclose(Ut @ Vt.T, (U @ V.T).T, rtol=0, atol=1e-12 * np.abs(M).max())
