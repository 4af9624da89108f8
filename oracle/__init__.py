"""FP64 CPU oracle for the HODLR direct solver (Chen & Martinsson, arXiv 2208.06290).

TEST INFRASTRUCTURE. This package is the independent reference that the CUDA
path is checked against. Only the test suite (``tests/``), the smoke check in
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs
of ``bench.py`` may import it. The product path (``paper_2208_06290_gb300``)
never imports it, and this package never imports the product path: the two
share no code. The only thing both sides consume is the seeded input
generator package ``synth``, which holds none of the method's arithmetic.

Contents
--------
``hodlr``
    * ``HodlrTree``: uniform cluster tree and the U_big/V_big column layout
      (Def. 1, Def. 2, Fig. 1, Eq. e:u, Fig. f:cat).
    * ``assemble_dense``: the N x N matrix a (D, U_big, V_big) triple
      represents (Eq. e:rank).
    * ``dense_*``: plain definitions on the assembled matrix (numpy LAPACK):
      solve, slogdet, adjoint solve, gradients of sum b^T A^-1 b + log|det A|.
    * ``RecursiveHODLR``: the recursive factor/solve of Sec. 3.1
      (Eqs. e:recursion, e:solution, e:node, Theorem 1), with the
      identity-diagonal coupling matrix of the variant after Alg. 4, the
      determinant by Sylvester's theorem (Sec. 3.5) and the adjoint solve by
      the same recursion on the transposed HODLR matrix.
    * ``matvec``: y = A x straight from the block definition.
    * ``sampled_rows_matvec``: individual rows of A x, for full-size checks.
``costs``
    The paper's closed-form storage / flop counts (Theorems t:store, t:solve
    and the factorization-cost theorem of Sec. 3.4) and the exact loop count
    of Alg. 1.

Parity status: every function here is pinned by ``tests/test_oracle.py``
against closed forms, dense LAPACK, brute-force element-wise assembly and
finite differences (see that file's module docstring for the list).
"""
