"""Storage and operation counts of the HODLR factor / solve (Sec. 3.4).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Two kinds of count:
* the paper's closed forms (Theorem t:store with the bullet reading
  mN + 2rNL, the factorization-cost theorem t_f and Theorem t:solve t_s);
* the exact count of the multiply-adds that Alg. 1 / Alg. 2 perform, written
  as a literal loop over levels and nodes, which the closed forms only
  approximate (the paper sums 4 r^2 N l over l = 1..L, while the loop over
  child levels c touches c-1 ancestor blocks).
"""
from __future__ import annotations


def paper_storage(N, m, r, L):
    """Entries of A: leaf blocks mN plus U_big and V_big 2rNL (Sec. 3.4 bullets)."""
    return m * N + 2 * r * N * L


def paper_factor_flops(N, m, r, L):
    """t_f = 2/3 m^2 N + 2 m r N L + 2 r^2 N (L + L^2) (factorization-cost theorem)."""
    return 2.0 / 3.0 * m * m * N + 2.0 * m * r * N * L + 2.0 * r * r * N * (L + L * L)


def paper_solve_flops(N, m, r, L):
    """t_s = 2 m N + 4 r N L per right-hand side (Theorem t:solve)."""
    return 2.0 * m * N + 4.0 * r * N * L


def loop_factor_flops(N, m, r, L):
    """Exact operation count of Alg. 1, walked node by node.

    Leaf stage: getrf of each m x m leaf (2/3 m^3) and getrs on its r*L
    right-hand-side columns (2 m^2 each). Level stage, children at level c
    (c = L .. 1), parents gamma at level c-1, child node size n = N / 2^c:
    * projections V^T Y over the own block and the c-1 ancestor blocks:
      2 n r (r c) per child;
    * LU of the 2r x 2r coupling matrix (2/3 (2r)^3) and its solve on
      r (c-1) right-hand sides (2 (2r)^2 each) per parent;
    * ancestor update Y(:, 1:r(c-1)) -= Y_own W: 2 n r (r (c-1)) per child.
    """
    total = 0.0
    nleaf = N // m
    for _ in range(nleaf):
        total += 2.0 / 3.0 * m ** 3 + 2.0 * m * m * (r * L)
    for c in range(L, 0, -1):
        n = N >> c
        anc = r * (c - 1)
        for _ in range(1 << (c - 1)):
            for _child in range(2):
                total += 2.0 * n * r * (r * c)
                total += 2.0 * n * r * anc
            total += 2.0 / 3.0 * (2 * r) ** 3 + 2.0 * (2 * r) ** 2 * anc
    return total


def loop_solve_flops(N, m, r, L, k=1):
    """Exact operation count of Alg. 2 for k right-hand sides: leaf getrs
    (2 m^2 per leaf per column), then per level the projections V^T x
    (2 n r), the coupling solve (2 (2r)^2 per parent) and the update Y w (2 n r)."""
    total = 0.0
    nleaf = N // m
    total += nleaf * 2.0 * m * m * k
    for c in range(L, 0, -1):
        n = N >> c
        for _ in range(1 << (c - 1)):
            total += 2 * (2.0 * n * r * k + 2.0 * n * r * k)
            total += 2.0 * (2 * r) ** 2 * k
    return total


def matvec_flops(N, m, r, L, k=1):
    """y = A x from the block definition: 2 m^2 per leaf, and per pair of
    siblings two V^T x products and two U (.) products of 2 n r each."""
    total = (N // m) * 2.0 * m * m * k
    for c in range(1, L + 1):
        n = N >> c
        total += (1 << (c - 1)) * 4 * (2.0 * n * r * k)
    return total
