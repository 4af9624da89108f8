"""Pins of the FP64 oracle against things other than itself (CPU only).

What fixes each oracle function:
* tree / layout: the index sets printed in Fig. 1 and the column layout of
  Fig. f:cat / Eq. e:u (golden fixtures under tests/golden/);
* ``assemble_dense``: an element-by-element brute-force assembly that finds,
  for every (i, j), the first level where i and j fall in different nodes;
* ``RecursiveHODLR.solve`` / ``slogdet`` / ``solve_adjoint``: the closed-form
  inverse and determinant of a 2 x 2 HODLR matrix (m = 1, L = 1, r = 1), the
  Sherman-Morrison closed form for one nonzero rank-1 block, the block-diagonal
  case (U = V = 0, per-leaf LAPACK), and dense LAPACK on the assembled matrix
  for random trees;
* the coupling matrix: its off-diagonal blocks equal V^T A_child^{-1} U from a
  dense solve of the child's assembled block (Theorem 1 / Eq. e:wood);
* the stored Y: the product A^(L+1) ... A^(1) of Sec. 3.5 rebuilds A;
* ``matvec`` / ``sampled_rows_matvec``: the assembled matrix times X;
* gradients: central finite differences of the dense loss, torch autograd of
  the dense loss, and the solve-based block formulas against the dense ones;
* cost counts: the closed forms printed in Sec. 3.4 (Theorems t:store, t:solve,
  factorization cost).
"""
import math
import os

import numpy as np
import pytest
import torch

from oracle import costs
from oracle.hodlr import (HodlrTree, RecursiveHODLR, assemble_dense, dense_grad,
                          dense_loss, dense_slogdet, dense_solve, dense_solve_adjoint,
                          grad_blocks, matvec, sampled_rows_matvec)
from synth import HodlrShape, gaussian_rhs, synthetic_hodlr, to_math

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(x) for x in line.split()])
    return rows


def _node_of_heap(h):
    c = h.bit_length() - 1
    return c, h - (1 << c)


def random_hodlr(N, L, r, seed, shift=4.0, k=2):
    D, U, V, g = synthetic_hodlr(HodlrShape(N, L, r), shift, seed)
    B = gaussian_rhs(N, k, g)
    return to_math(D, U, V, B)


# ---------------------------------------------------------------- tree / layout
def test_fig1_index_sets():
    t = HodlrTree(400, 2, 1)
    for h, first, last in _read_golden("fig1_index_sets.txt"):
        c, i = _node_of_heap(h)
        assert HodlrTree.heap_number(c, i) == h
        s = t.rows(c, i)
        assert (s.start + 1, s.stop) == (first, last)


def test_fig_cat_layout():
    r = 3
    t = HodlrTree(400, 2, r)
    for h, block, first, last in _read_golden("fig_cat_layout.txt"):
        c, i = _node_of_heap(h)
        cs = t.cols(c)
        assert (cs.start, cs.stop) == ((block - 1) * r, block * r)
        s = t.rows(c, i)
        assert (s.start + 1, s.stop) == (first, last)


def _bruteforce_entry(D, U, V, L, i, j):
    N = U.shape[0]
    m = N >> L
    r = U.shape[1] // L
    if i // m == j // m:
        return D[i // m][i % m, j % m]
    c = next(c for c in range(1, L + 1) if i // (N >> c) != j // (N >> c))
    # i's node and j's node at level c are siblings; A(i, j) = U_i-node(i,:) . V_j-node(j,:)
    cols = slice((c - 1) * r, c * r)
    return float(U[i, cols] @ V[j, cols])


@pytest.mark.parametrize("N,L,r", [(8, 2, 1), (24, 3, 2), (32, 2, 4)])
def test_assemble_bruteforce(N, L, r):
    D, U, V, _ = random_hodlr(N, L, r, seed=3)
    A = assemble_dense(D, U, V, L)
    B = np.array([[_bruteforce_entry(D, U, V, L, i, j) for j in range(N)] for i in range(N)])
    np.testing.assert_array_equal(A, B)


# ---------------------------------------------------------------- closed forms
def test_scalar_2x2_closed_form():
    """m = 1, L = 1, r = 1: A = [[d1, u1 v2], [u2 v1, d2]]."""
    d1, d2, u1, u2, v1, v2 = 1.7, -0.9, 0.3, -1.1, 0.8, 0.45
    D = np.array([[[d1]], [[d2]]])
    U = np.array([[u1], [u2]])
    V = np.array([[v1], [v2]])
    det = d1 * d2 - u1 * v2 * u2 * v1
    b = np.array([[0.25], [-2.0]])
    x_true = np.array([[d2 * b[0, 0] - u1 * v2 * b[1, 0]],
                       [-u2 * v1 * b[0, 0] + d1 * b[1, 0]]]) / det
    xt_true = np.array([[d2 * b[0, 0] - u2 * v1 * b[1, 0]],
                        [-u1 * v2 * b[0, 0] + d1 * b[1, 0]]]) / det
    rec = RecursiveHODLR(D, U, V, 1)
    np.testing.assert_allclose(rec.solve(b), x_true, rtol=1e-14)
    np.testing.assert_allclose(rec.solve_adjoint(b), xt_true, rtol=1e-14)
    s, la = rec.slogdet()
    assert s == np.sign(det)
    assert la == pytest.approx(math.log(abs(det)), rel=1e-14)


def test_sherman_morrison_one_block():
    """L = 1, rank 1, U_beta = 0: A = blockdiag(D1, D2) + [u1; 0][0; v2]^T, so
    x = D^{-1} b - [D1^{-1} u1 (v2^T D2^{-1} b2); 0] and det A = det D1 det D2."""
    rng = np.random.default_rng(7)
    m = 5
    D = rng.standard_normal((2, m, m)) + 3 * np.eye(m)
    U = np.zeros((2 * m, 1))
    V = np.zeros((2 * m, 1))
    U[:m, 0] = rng.standard_normal(m)          # u1 = U_alpha
    V[m:, 0] = rng.standard_normal(m)          # v2 = V_beta
    V[:m, 0] = rng.standard_normal(m)          # V_alpha: multiplies U_beta = 0
    b = rng.standard_normal((2 * m, 1))
    D1i_b1 = np.linalg.solve(D[0], b[:m])
    D2i_b2 = np.linalg.solve(D[1], b[m:])
    D1i_u1 = np.linalg.solve(D[0], U[:m])
    x_true = np.concatenate([D1i_b1 - D1i_u1 * float(V[m:, 0] @ D2i_b2[:, 0]), D2i_b2])
    rec = RecursiveHODLR(D, U, V, 1)
    np.testing.assert_allclose(rec.solve(b), x_true, rtol=1e-12, atol=1e-13)
    s1, l1 = np.linalg.slogdet(D[0])
    s2, l2 = np.linalg.slogdet(D[1])
    s, la = rec.slogdet()
    assert s == s1 * s2
    assert la == pytest.approx(l1 + l2, rel=1e-13, abs=1e-13)


def test_block_diagonal():
    rng = np.random.default_rng(11)
    L, m, r = 3, 4, 2
    N = m << L
    D = rng.standard_normal((1 << L, m, m)) + 2 * np.eye(m)
    U = np.zeros((N, r * L))
    V = np.zeros((N, r * L))
    B = rng.standard_normal((N, 3))
    rec = RecursiveHODLR(D, U, V, L)
    x = rec.solve(B)
    for b in range(1 << L):
        s = slice(b * m, (b + 1) * m)
        np.testing.assert_allclose(x[s], np.linalg.solve(D[b], B[s]), rtol=1e-12)
    s, la = rec.slogdet()
    ref = [np.linalg.slogdet(D[b]) for b in range(1 << L)]
    assert s == np.prod([q[0] for q in ref])
    assert la == pytest.approx(sum(q[1] for q in ref), rel=1e-13)


# ---------------------------------------------------------------- vs dense LAPACK
CASES = [(16, 1, 2), (64, 3, 3), (96, 2, 5), (256, 4, 4), (512, 3, 8)]


@pytest.mark.parametrize("N,L,r", CASES)
def test_recursive_vs_dense(N, L, r):
    D, U, V, B = random_hodlr(N, L, r, seed=N + L + r)
    rec = RecursiveHODLR(D, U, V, L)
    A = assemble_dense(D, U, V, L)
    x = rec.solve(B)
    np.testing.assert_allclose(x, np.linalg.solve(A, B), rtol=1e-10, atol=1e-12)
    assert np.linalg.norm(B - A @ x) / np.linalg.norm(B) < 1e-13
    np.testing.assert_allclose(rec.solve_adjoint(B), np.linalg.solve(A.T, B), rtol=1e-10, atol=1e-12)
    s, la = rec.slogdet()
    sd, lad = np.linalg.slogdet(A)
    assert s == sd
    assert la == pytest.approx(lad, rel=1e-12, abs=1e-11)
    assert dense_slogdet(D, U, V, L)[1] == pytest.approx(lad, rel=1e-14)
    np.testing.assert_allclose(dense_solve(D, U, V, L, B), np.linalg.solve(A, B), rtol=1e-12)
    np.testing.assert_allclose(dense_solve_adjoint(D, U, V, L, B), np.linalg.solve(A.T, B), rtol=1e-12)


def test_negative_determinant_sign():
    """A leaf with one negative eigenvalue direction flips the sign of det A."""
    D, U, V, B = random_hodlr(64, 2, 2, seed=5)
    U, V = 0.1 * U, 0.1 * V
    D[1][0] *= -1.0          # one leaf row negated: det D_1 changes sign
    rec = RecursiveHODLR(D, U, V, 2)
    sd, lad = np.linalg.slogdet(assemble_dense(D, U, V, 2))
    s, la = rec.slogdet()
    assert sd == -1.0
    assert s == sd
    assert la == pytest.approx(lad, rel=1e-12)


def test_symmetric_adjoint_equals_solve():
    D, U, V, B = random_hodlr(128, 3, 3, seed=2)
    D = 0.5 * (D + np.transpose(D, (0, 2, 1)))
    V = U.copy()
    rec = RecursiveHODLR(D, U, V, 3)
    np.testing.assert_allclose(rec.solve_adjoint(B), rec.solve(B), rtol=1e-12, atol=1e-13)


def test_coupling_is_capacitance_matrix():
    """Theorem 1 / Eq. e:wood: the off-diagonal blocks of K~ at the root are
    V_beta^T A_beta^{-1} U_beta and V_alpha^T A_alpha^{-1} U_alpha, with A_child the
    child's diagonal block of the assembled matrix, solved densely."""
    N, L, r = 128, 3, 3
    D, U, V, _ = random_hodlr(N, L, r, seed=9)
    A = assemble_dense(D, U, V, L)
    t = HodlrTree(N, L, r)
    rec = RecursiveHODLR(D, U, V, L)
    K = rec.node_coupling(0, 0)
    ra, rb = t.rows(1, 0), t.rows(1, 1)
    Ta = t.V_node(V, 1, 0).T @ np.linalg.solve(A[ra, ra], t.U_node(U, 1, 0))
    Tb = t.V_node(V, 1, 1).T @ np.linalg.solve(A[rb, rb], t.U_node(U, 1, 1))
    np.testing.assert_allclose(K[:r, r:], Tb, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(K[r:, :r], Ta, rtol=1e-12, atol=1e-14)
    np.testing.assert_array_equal(K[:r, :r], np.eye(r))
    np.testing.assert_array_equal(K[r:, r:], np.eye(r))


def test_factorization_reconstructs_A():
    """Sec. 3.5: A = A^(L+1) A^(L) ... A^(1), A^(L+1) = blockdiag(D_b), and the
    level-c factor is blockdiag over parents of I + [[0, Y_a V_b^T], [Y_b V_a^T, 0]]."""
    N, L, r = 64, 3, 2
    D, U, V, _ = random_hodlr(N, L, r, seed=4)
    t = HodlrTree(N, L, r)
    rec = RecursiveHODLR(D, U, V, L)
    P = np.zeros((N, N))
    for b in range(1 << L):
        s = t.rows(L, b)
        P[s, s] = D[b]
    for c in range(L, 0, -1):
        F = np.eye(N)
        for j in range(1 << (c - 1)):
            a, b = (c, 2 * j), (c, 2 * j + 1)
            ra, rb = t.rows(*a), t.rows(*b)
            F[ra, rb] = rec.Y[a] @ t.V_node(V, *b).T
            F[rb, ra] = rec.Y[b] @ t.V_node(V, *a).T
        P = P @ F
    np.testing.assert_allclose(P, assemble_dense(D, U, V, L), rtol=1e-12, atol=1e-13)


# ---------------------------------------------------------------- matvec
@pytest.mark.parametrize("N,L,r", [(64, 3, 3), (256, 4, 4)])
def test_matvec(N, L, r):
    D, U, V, B = random_hodlr(N, L, r, seed=1)
    A = assemble_dense(D, U, V, L)
    np.testing.assert_allclose(matvec(D, U, V, L, B), A @ B, rtol=1e-12, atol=1e-13)
    rows = [0, 5, N // 2, N - 1]
    np.testing.assert_allclose(sampled_rows_matvec(D, U, V, L, B, rows), (A @ B)[rows],
                               rtol=1e-12, atol=1e-13)


# ---------------------------------------------------------------- gradients
def _flat(D, U, V, B):
    return np.concatenate([D.ravel(), U.ravel(), V.ravel(), B.ravel()])


def test_dense_grad_finite_differences():
    N, L, r = 32, 2, 2
    D, U, V, B = random_hodlr(N, L, r, seed=6)
    dD, dU, dV, dB = dense_grad(D, U, V, L, B)
    g = _flat(dD, dU, dV, dB)
    rng = np.random.default_rng(0)
    sizes = [D.size, U.size, V.size, B.size]
    for _ in range(5):
        d = rng.standard_normal(g.size)
        parts = np.split(d, np.cumsum(sizes)[:-1])
        dd = [p.reshape(x.shape) for p, x in zip(parts, (D, U, V, B))]
        h = 1e-6
        fp = dense_loss(D + h * dd[0], U + h * dd[1], V + h * dd[2], L, B + h * dd[3])
        fm = dense_loss(D - h * dd[0], U - h * dd[1], V - h * dd[2], L, B - h * dd[3])
        fd = (fp - fm) / (2 * h)
        assert fd == pytest.approx(float(g @ d), rel=1e-6)


def test_dense_grad_vs_torch_autograd_on_A():
    """d loss / d A = -Lam X^T + A^{-T} against torch autograd of the same loss."""
    N, L, r = 48, 2, 3
    D, U, V, B = random_hodlr(N, L, r, seed=8)
    A = torch.tensor(assemble_dense(D, U, V, L), requires_grad=True)
    Bt = torch.tensor(B, requires_grad=True)
    loss = (Bt * torch.linalg.solve(A, Bt)).sum() + torch.linalg.slogdet(A)[1]
    loss.backward()
    An = A.detach().numpy()
    X = np.linalg.solve(An, B)
    Lam = np.linalg.solve(An.T, B)
    G = -Lam @ X.T + np.linalg.inv(An).T
    np.testing.assert_allclose(A.grad.numpy(), G, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(Bt.grad.numpy(), dense_grad(D, U, V, L, B)[3], rtol=1e-10)


def test_grad_blocks_match_dense():
    N, L, r = 64, 3, 2
    D, U, V, B = random_hodlr(N, L, r, seed=12)
    dD, dU, dV, dB = dense_grad(D, U, V, L, B)
    t = HodlrTree(N, L, r)
    rec = RecursiveHODLR(D, U, V, L)
    pairs = [(1, 0), (1, 1), (2, 2), (3, 5)]
    got = grad_blocks(rec, B, leaves=[0, 6], pairs=pairs)
    np.testing.assert_allclose(got["B"], dB, rtol=1e-11, atol=1e-12)
    for b in (0, 6):
        np.testing.assert_allclose(got[("D", b)], dD[b], rtol=1e-10, atol=1e-12)
    for c, a in pairs:
        np.testing.assert_allclose(got[("U", c, a)], dU[t.rows(c, a), t.cols(c)], rtol=1e-10, atol=1e-12)
        s = a ^ 1
        np.testing.assert_allclose(got[("V", c, s)], dV[t.rows(c, s), t.cols(c)], rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------- costs
@pytest.mark.parametrize("N,m,r,L", [(4096, 64, 16, 6), (1 << 12, 128, 8, 5), (1 << 14, 256, 32, 6)])
def test_costs_match_paper_closed_forms(N, m, r, L):
    assert costs.paper_storage(N, m, r, L) == m * N + 2 * r * N * L
    coupling_solve = 8.0 * r * r * ((1 << L) - 1)
    assert costs.loop_solve_flops(N, m, r, L) - coupling_solve == pytest.approx(
        costs.paper_solve_flops(N, m, r, L), rel=1e-14)
    # The paper sums 4 r^2 N l over l = 1..L (= 2 r^2 N (L + L^2)); the loop over
    # child levels c has 2 r^2 N (2c - 1) per level (= 2 r^2 N L^2) plus the
    # 2r x 2r coupling LUs and solves.
    coupling = sum((1 << (c - 1)) * (2.0 / 3.0 * (2 * r) ** 3 + 2.0 * (2 * r) ** 2 * r * (c - 1))
                   for c in range(1, L + 1))
    assert costs.loop_factor_flops(N, m, r, L) - coupling == pytest.approx(
        costs.paper_factor_flops(N, m, r, L) - 2.0 * r * r * N * L, rel=1e-12)
    assert costs.matvec_flops(N, m, r, L) == pytest.approx(2 * costs.paper_storage(N, m, r, L), rel=1e-14)


def test_generator_layout_and_determinism():
    s = HodlrShape(256, 2, 4)
    D1, U1, V1, g1 = synthetic_hodlr(s, 4.0, 123)
    D2, U2, V2, g2 = synthetic_hodlr(s, 4.0, 123)
    assert torch.equal(D1, D2) and torch.equal(U1, U2) and torch.equal(V1, V2)
    assert D1.stride() == (64 * 64, 1, 64)
    assert U1.stride() == (1, 256) and U1.shape == (256, 8)
    # level scales 0.5/sqrt(n_c)
    assert U1[:, :4].std().item() == pytest.approx(0.5 / math.sqrt(128), rel=0.15)
    assert U1[:, 4:].std().item() == pytest.approx(0.5 / math.sqrt(64), rel=0.15)
