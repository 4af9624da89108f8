"""Seeded synthetic inputs for the HODLR solver.

This package only draws random numbers and lays them out; it holds none of
the solver's arithmetic (no factorization, solve, determinant or product with
the HODLR operator). Both the CUDA path (tests, bench) and the FP64 oracle read
the tensors it returns, so that the two sides see identical inputs.
"""
from .generators import (  # noqa: F401
    HodlrShape,
    synthetic_hodlr,
    gaussian_rhs,
    to_math,
)
