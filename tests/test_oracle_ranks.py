"""Pin of the oracle's assembly of a HODLR matrix with per-level ranks in the
ragged layout (Eq. e:u with per-level widths; CPU only): every entry against
a brute-force formula that finds, for (i, j) in different leaves, the level
c where i and j first fall in different nodes and sums the r_c products of
their level-c basis rows."""
import numpy as np

from oracle.hodlr import assemble_dense_level_ranks


def test_level_rank_assembly_brute_force():
    rng = np.random.default_rng(4)
    N, L = 64, 3
    m = N >> L
    ranks = [3, 1, 2]
    D = rng.standard_normal((1 << L, m, m))
    Ur = rng.standard_normal((N, sum(ranks)))
    Vr = rng.standard_normal((N, sum(ranks)))
    A = assemble_dense_level_ranks(D, Ur, Vr, L, ranks)
    off = np.cumsum([0] + ranks)
    for i in range(N):
        for j in range(N):
            if i // m == j // m:
                want = D[i // m][i % m, j % m]
            else:
                c = next(c for c in range(1, L + 1) if i // (N >> c) != j // (N >> c))
                cols = slice(off[c - 1], off[c])
                want = Ur[i, cols] @ Vr[j, cols]
            assert A[i, j] == want
