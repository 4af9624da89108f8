"""Plain FP64 CPU oracle of the HODLR factor / solve / logdet / adjoint / gradient.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): never imported by the
product path; imports nothing from it.

Conventions (all arrays float64, numpy, "math" indexing)
--------------------------------------------------------
* ``D``: shape (2^L, m, m); ``D[b]`` is the leaf block A(I_b, I_b) of leaf b
  (leaves numbered left to right, leaf b owns rows b*m .. b*m+m-1).
* ``U``, ``V``: shape (N, r*L); column block j (columns j*r .. j*r+r-1) holds
  the bases of the tree nodes at level j+1, each on its own rows, parent
  levels to the left (Eq. e:u, Fig. f:cat).
* Node (c, i) is node i (0-based, left to right) at level c; its heap number
  in Fig. 1 is 2^c + i. Its rows are I_(c,i) = [i*N/2^c, (i+1)*N/2^c).
* The off-diagonal block between siblings alpha=(c,2j), beta=(c,2j+1) is
  A(I_alpha, I_beta) = U_alpha V_beta^T and A(I_beta, I_alpha) = U_beta V_alpha^T
  (Eq. e:rank), with U_alpha = U(I_alpha, block c-1), V_beta = V(I_beta, block c-1).

Readings of the paper taken here (each also listed in the design notes):
* Coupling matrix: the identity-diagonal variant given after Alg. 4,
  K~ = [[I, V_beta^T Y_beta], [V_alpha^T Y_alpha, I]] with right-hand side
  [V_beta^T z_beta; V_alpha^T z_alpha] and unknowns [w_alpha; w_beta]. It has
  the same solution as Eq. e:node (rows swapped) and det K~ = det of the
  2x2-block factor of Sec. 3.5 with no sign change.
* Real field only (F = R).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


# --------------------------------------------------------------------------
# Tree and layout (Def. 1, Def. 2, Fig. 1, Eq. e:u)
# --------------------------------------------------------------------------
class HodlrTree:
    """Uniform cluster tree T_L of Def. 1: levels 0..L, 2^c nodes at level c,
    consecutive index sets, leaves of size m, N = m * 2^L."""

    def __init__(self, N: int, L: int, r: int):
        if L < 0 or N % (1 << L) != 0:
            raise ValueError("N must be m * 2^L")
        self.N, self.L, self.r = N, L, r
        self.m = N >> L

    def rows(self, c: int, i: int) -> slice:
        """Index set I_(c,i) of node i at level c (0-based, half-open)."""
        n = self.N >> c
        return slice(i * n, (i + 1) * n)

    def cols(self, c: int) -> slice:
        """Columns of U_big / V_big holding the level-c bases (Eq. e:u)."""
        if not 1 <= c <= self.L:
            raise ValueError("bases exist for levels 1..L")
        return slice((c - 1) * self.r, c * self.r)

    @staticmethod
    def heap_number(c: int, i: int) -> int:
        """Heap numbering of Fig. 1: root 1, children of gamma are 2gamma, 2gamma+1."""
        return (1 << c) + i

    def U_node(self, U, c, i):
        return U[self.rows(c, i), self.cols(c)]

    def V_node(self, V, c, i):
        return V[self.rows(c, i), self.cols(c)]


def _check(D, U, V, L):
    nleaf, m, m2 = D.shape
    if m != m2 or nleaf != (1 << L):
        raise ValueError("D must have shape (2^L, m, m)")
    N = nleaf * m
    if U.shape != V.shape or U.shape[0] != N or (L > 0 and U.shape[1] % L):
        raise ValueError("U, V must have shape (N, r*L)")
    r = U.shape[1] // L if L > 0 else 0
    return HodlrTree(N, L, r)


# --------------------------------------------------------------------------
# Dense tier: the plain definitions on the assembled matrix
# --------------------------------------------------------------------------
def assemble_dense(D, U, V, L) -> np.ndarray:
    """The N x N matrix represented by (D, U_big, V_big): leaf blocks on the
    diagonal (Fig. 2) and A(I_alpha, I_beta) = U_alpha V_beta^T for every pair of
    siblings (Eq. e:rank)."""
    t = _check(D, U, V, L)
    A = np.zeros((t.N, t.N))
    for b in range(1 << L):
        s = t.rows(L, b)
        A[s, s] = D[b]
    for c in range(1, L + 1):
        for j in range(1 << (c - 1)):
            a, b = 2 * j, 2 * j + 1
            ra, rb = t.rows(c, a), t.rows(c, b)
            A[ra, rb] = t.U_node(U, c, a) @ t.V_node(V, c, b).T
            A[rb, ra] = t.U_node(U, c, b) @ t.V_node(V, c, a).T
    return A


def dense_solve(D, U, V, L, B):
    """x = A^{-1} B by LAPACK on the assembled matrix."""
    return np.linalg.solve(assemble_dense(D, U, V, L), B)


def dense_solve_adjoint(D, U, V, L, B):
    """x = A^{-T} B by LAPACK on the assembled matrix."""
    return np.linalg.solve(assemble_dense(D, U, V, L).T, B)


def dense_slogdet(D, U, V, L):
    """(sign, log|det A|) by LAPACK on the assembled matrix."""
    return np.linalg.slogdet(assemble_dense(D, U, V, L))


def dense_loss(D, U, V, L, B) -> float:
    """loss = sum_j b_j^T A^{-1} b_j + log|det A| on the assembled matrix."""
    A = assemble_dense(D, U, V, L)
    X = np.linalg.solve(A, B)
    return float(np.sum(B * X) + np.linalg.slogdet(A)[1])


def grad_from_dense_G(G, t: HodlrTree, U, V):
    """Chain a gradient G = d loss / d A (N x N) to the HODLR parameters.

    A(I_b, I_b) = D_b gives dD_b = G(I_b, I_b); A(I_alpha, I_beta) = U_alpha V_beta^T
    gives dU_alpha = G(I_alpha, I_beta) V_beta and dV_beta = G(I_alpha, I_beta)^T U_alpha.
    Every U_alpha and V_beta appears in exactly one block, so these are complete.
    """
    L = t.L
    dD = np.stack([G[t.rows(L, b), t.rows(L, b)] for b in range(1 << L)])
    dU = np.zeros_like(U)
    dV = np.zeros_like(V)
    for c in range(1, L + 1):
        for j in range(1 << (c - 1)):
            for a, b in ((2 * j, 2 * j + 1), (2 * j + 1, 2 * j)):
                ra, rb = t.rows(c, a), t.rows(c, b)
                cc = t.cols(c)
                dU[ra, cc] = G[ra, rb] @ V[rb, cc]
                dV[rb, cc] = G[ra, rb].T @ U[ra, cc]
    return dD, dU, dV


def dense_grad(D, U, V, L, B):
    """Gradients of loss = sum_j b_j^T A^{-1} b_j + log|det A|.

    Matrix calculus on the assembled A: with X = A^{-1} B and Lam = A^{-T} B,
    d/dB = X + Lam and d/dA = -Lam X^T + A^{-T}; then chained to D, U, V by
    ``grad_from_dense_G``. Returns (dD, dU, dV, dB).
    """
    t = _check(D, U, V, L)
    A = assemble_dense(D, U, V, L)
    X = np.linalg.solve(A, B)
    Lam = np.linalg.solve(A.T, B)
    G = -Lam @ X.T + np.linalg.inv(A).T
    dD, dU, dV = grad_from_dense_G(G, t, U, V)
    return dD, dU, dV, X + Lam


# --------------------------------------------------------------------------
# Operator application straight from the definition
# --------------------------------------------------------------------------
def matvec(D, U, V, L, X):
    """Y = A X without forming A: leaf blocks plus, for every pair of
    siblings, U_alpha (V_beta^T X_beta) and U_beta (V_alpha^T X_alpha) (Eq. e:rank)."""
    t = _check(D, U, V, L)
    X = np.asarray(X, dtype=np.float64)
    Y = np.zeros_like(X)
    for b in range(1 << L):
        s = t.rows(L, b)
        Y[s] = D[b] @ X[s]
    for c in range(1, L + 1):
        for j in range(1 << (c - 1)):
            a, b = 2 * j, 2 * j + 1
            ra, rb = t.rows(c, a), t.rows(c, b)
            Y[ra] += t.U_node(U, c, a) @ (t.V_node(V, c, b).T @ X[rb])
            Y[rb] += t.U_node(U, c, b) @ (t.V_node(V, c, a).T @ X[ra])
    return Y


def sampled_rows_matvec(D, U, V, L, X, rows):
    """Rows ``rows`` of A X, each computed on its own from row i of A: the
    leaf-block row D_b(i, :) X(I_b) plus, for every level c, the basis row
    U_alpha(i, :) times V_beta^T X(I_beta) where alpha is i's node at level c and
    beta its sibling. Lets a full-size product be checked one row at a time."""
    t = _check(D, U, V, L)
    X = np.asarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    out = np.zeros((len(rows), X.shape[1]))
    for k, i in enumerate(rows):
        b = i // t.m
        s = t.rows(L, b)
        acc = D[b][i - s.start] @ X[s]
        for c in range(1, L + 1):
            a = i // (t.N >> c)
            sib = a ^ 1
            cc = t.cols(c)
            acc = acc + U[i, cc] @ (V[t.rows(c, sib), cc].T @ X[t.rows(c, sib)])
        out[k] = acc
    return out


# --------------------------------------------------------------------------
# Recursive tier (Sec. 3.1: Eqs. e:recursion, e:solution, e:node; Theorem 1)
# --------------------------------------------------------------------------
class RecursiveHODLR:
    """Recursive HODLR factorization and solve, in FP64.

    Factorization stage (end of Sec. 3.1): for every internal node gamma with
    children alpha, beta, compute Y_alpha = A_alpha^{-1} U_alpha and
    Y_beta = A_beta^{-1} U_beta by the recursion itself, then an LU factorization of
    the coupling matrix K~_gamma = [[I, V_beta^T Y_beta], [V_alpha^T Y_alpha, I]].
    Leaves keep an LU factorization (partial pivoting, LAPACK getrf) of D_b.

    Solution stage: A_gamma^{-1} b = [z_alpha - Y_alpha w_alpha; z_beta - Y_beta w_beta]
    with z = A_child^{-1} b_child (Eq. e:recursion), and
    K~ [w_alpha; w_beta] = [V_beta^T z_beta; V_alpha^T z_alpha] (Eq. e:node, rows
    swapped to the identity-diagonal form).

    Determinant (Sec. 3.5): A = A^(L+1) ... A^(1) with A^(L+1) = blockdiag(D_b)
    and each 2x2-block factor I + [[0, Y_alpha V_beta^T], [Y_beta V_alpha^T, 0]]
    whose determinant equals det K~_gamma by Sylvester's theorem, so
    log|det A| = sum_b log|det D_b| + sum_gamma log|det K~_gamma|.
    """

    def __init__(self, D, U, V, L):
        self.t = _check(D, U, V, L)
        self.D, self.U, self.V, self.L = D, U, V, L
        self.leaf_lu = {}
        self.Y = {}
        self.K = {}
        self.K_lu = {}
        self._factor(0, 0)

    # -- factorization stage -------------------------------------------------
    def _factor(self, c, i):
        t, L = self.t, self.L
        if c == L:
            self.leaf_lu[i] = sla.lu_factor(self.D[i], check_finite=True)
            return
        a, b = (c + 1, 2 * i), (c + 1, 2 * i + 1)
        self._factor(*a)
        self._factor(*b)
        Ya = self.apply_inverse(a, t.U_node(self.U, *a))
        Yb = self.apply_inverse(b, t.U_node(self.U, *b))
        Va, Vb = t.V_node(self.V, *a), t.V_node(self.V, *b)
        r = t.r
        K = np.eye(2 * r)
        K[:r, r:] = Vb.T @ Yb
        K[r:, :r] = Va.T @ Ya
        self.Y[a], self.Y[b] = Ya, Yb
        self.K[(c, i)] = K
        self.K_lu[(c, i)] = sla.lu_factor(K, check_finite=True)

    # -- solution stage ------------------------------------------------------
    def apply_inverse(self, node, B):
        """A_node^{-1} B for the sub-HODLR matrix of ``node`` (Eqs. e:recursion,
        e:solution, e:node)."""
        c, i = node
        t, L, r = self.t, self.L, self.t.r
        if c == L:
            return sla.lu_solve(self.leaf_lu[i], B)
        a, b = (c + 1, 2 * i), (c + 1, 2 * i + 1)
        half = B.shape[0] // 2
        Za = self.apply_inverse(a, B[:half])
        Zb = self.apply_inverse(b, B[half:])
        Va, Vb = t.V_node(self.V, *a), t.V_node(self.V, *b)
        rhs = np.concatenate([Vb.T @ Zb, Va.T @ Za], axis=0)
        w = sla.lu_solve(self.K_lu[node], rhs)
        return np.concatenate([Za - self.Y[a] @ w[:r], Zb - self.Y[b] @ w[r:]], axis=0)

    def solve(self, B):
        """x = A^{-1} B."""
        return self.apply_inverse((0, 0), np.asarray(B, dtype=np.float64))

    def slogdet(self):
        """(sign, log|det A|) by the factorization of Sec. 3.5."""
        sign, logabs = 1.0, 0.0
        for b in range(1 << self.L):
            s, la = np.linalg.slogdet(self.D[b])
            sign *= s
            logabs += la
        for K in self.K.values():
            s, la = np.linalg.slogdet(K)
            sign *= s
            logabs += la
        return sign, logabs

    def transposed(self) -> "RecursiveHODLR":
        """Factorization of A^T. A^T(I_alpha, I_beta) = (U_beta V_alpha^T)^T = V_alpha U_beta^T,
        so A^T is the HODLR matrix with leaf blocks D_b^T and the roles of U and V
        exchanged."""
        return RecursiveHODLR(np.ascontiguousarray(np.transpose(self.D, (0, 2, 1))),
                              self.V, self.U, self.L)

    def solve_adjoint(self, B):
        """x = A^{-T} B via the recursion on the transposed HODLR matrix."""
        return self.transposed().solve(B)

    def node_coupling(self, c, i):
        """K~ of node (c, i) (c < L)."""
        return self.K[(c, i)]


# --------------------------------------------------------------------------
# Gradients at any size, one block at a time (sampled checks of big problems)
# --------------------------------------------------------------------------
def embed(t: HodlrTree, rows: slice, M):
    """N x k matrix equal to M on ``rows`` and zero elsewhere."""
    out = np.zeros((t.N, M.shape[1]))
    out[rows] = M
    return out


def grad_blocks(rec: RecursiveHODLR, B, leaves=(), pairs=()):
    """Selected gradient blocks of loss = sum_j b_j^T A^{-1} b_j + log|det A|,
    from G = -Lam X^T + A^{-T} (Lam = A^{-T} B, X = A^{-1} B), evaluated through
    solves only, so that it runs at any N:

    * dD_b = G(I_b, I_b) = -Lam_b X_b^T + (A^{-1} E_b)(I_b)^T, with E_b the
      columns of the identity on I_b (m solves);
    * for a pair (c, a) with sibling s: dU_a = G(I_a, I_s) V_s
      = -Lam_a (X_s^T V_s) + (A^{-T} embed(V_s))(I_a)            (r adjoint solves)
      dV_s = G(I_a, I_s)^T U_a = -X_s (Lam_a^T U_a) + (A^{-1} embed(U_a))(I_s)  (r solves).

    Returns dict with keys ('D', b), ('U', c, a), ('V', c, s) and 'B'.
    """
    t = rec.t
    recT = rec.transposed()
    X = rec.solve(B)
    Lam = recT.solve(B)
    out = {"B": X + Lam}
    for b in leaves:
        s = t.rows(t.L, b)
        E = embed(t, s, np.eye(t.m))
        out[("D", b)] = -Lam[s] @ X[s].T + rec.solve(E)[s].T
    for c, a in pairs:
        sib = a ^ 1
        ra, rs = t.rows(c, a), t.rows(c, sib)
        Ua, Vs = t.U_node(rec.U, c, a), t.V_node(rec.V, c, sib)
        out[("U", c, a)] = -Lam[ra] @ (X[rs].T @ Vs) + recT.solve(embed(t, rs, Vs))[ra]
        out[("V", c, sib)] = -X[rs] @ (Lam[ra].T @ Ua) + rec.solve(embed(t, ra, Ua))[rs]
    return out


# --------------------------------------------------------------------------
# Construction (Sec. 2.2): partial-pivoted cross approximation of one block
# --------------------------------------------------------------------------
def cross_approximation(M, r, rows=None, cols=None):
    """Rank-r partial-pivoted cross approximation of the dense block M
    (n x n'), in FP64: i_0 = 0; for k = 0 .. r-1 the residual row
    rho = M(i_k, :) - sum_{l<k} u_l(i_k) v_l, its largest entry among unused
    columns j_k (first maximum), v_k = rho / rho(j_k), the residual column
    u_k = M(:, j_k) - sum_{l<k} v_l(j_k) u_l, and i_{k+1} the largest entry of
    |u_k| among unused rows (first maximum). A vanishing residual ends the
    approximation (remaining columns zero). With `rows`, `cols` given (pivot
    sequences, -1 = ended), those pivots are taken instead of the maxima.
    Returns (U (n x r), V (n' x r), rows, cols) with M ~= U V^T."""
    M = np.asarray(M, dtype=np.float64)
    n, n2 = M.shape
    U = np.zeros((n, r))
    V = np.zeros((n2, r))
    prow, pcol = [], []
    i = 0
    for k in range(r):
        if rows is not None:
            i = rows[k]
        if i < 0:
            break
        prow.append(i)
        rho = M[i, :] - U[i, :k] @ V[:, :k].T
        if cols is not None:
            j = cols[k]
            if j < 0:
                break
        else:
            a = np.abs(rho)
            a[pcol] = -1.0
            j = int(np.argmax(a))
            if rho[j] == 0.0:
                break
        pcol.append(j)
        V[:, k] = rho / rho[j]
        U[:, k] = M[:, j] - U[:, :k] @ V[j, :k]
        a = np.abs(U[:, k])
        a[prow] = -1.0
        i = int(np.argmax(a))
        if a[i] <= 0.0:
            i = -1
    return U, V, prow, pcol


def assemble_dense_level_ranks(D, Ur, Vr, L, level_ranks):
    """The N x N matrix of a HODLR matrix with per-level ranks r_c in the
    ragged layout (level c's bases in columns sum(r_1..r_{c-1}) .. + r_c - 1):
    leaf blocks on the diagonal and A(I_alpha, I_beta) = U_alpha V_beta^T with
    U_alpha, V_beta the r_c-column blocks of their level (Eq. e:rank)."""
    nleaf, m, _ = D.shape
    N = nleaf * m
    A = np.zeros((N, N))
    for b in range(nleaf):
        A[b * m:(b + 1) * m, b * m:(b + 1) * m] = D[b]
    off = 0
    for c in range(1, L + 1):
        n = N >> c
        cols = slice(off, off + level_ranks[c - 1])
        for j in range(1 << (c - 1)):
            a, b = 2 * j, 2 * j + 1
            ra, rb = slice(a * n, (a + 1) * n), slice(b * n, (b + 1) * n)
            A[ra, rb] = Ur[ra, cols] @ Vr[rb, cols].T
            A[rb, ra] = Ur[rb, cols] @ Vr[ra, cols].T
        off += level_ranks[c - 1]
    return A
