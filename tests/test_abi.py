"""Host-side checks of the C ABI (no GPU): the library builds and loads, every
function include/hodlr.h declares is exported, host argument validation, and
the product's closed-form cost counts against the oracle's loop counts."""
import ctypes
import os
import re

import pytest
import torch

from oracle import costs as ocosts

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hodlr.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hodlr_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def hb():
    from paper_2208_06290_gb300 import binding
    return binding


def test_every_declared_symbol_is_exported(hb):
    names = _declared()
    assert len(names) >= 14
    lib = ctypes.CDLL(hb._build.LIB)
    for n in names:
        assert hasattr(lib, n), n
    assert set(hb.EXPORTED) == set(names)


def test_strerror(hb):
    assert hb._strerror(0) == "ok"
    assert "singular" in hb._strerror(hb.HODLR_ERR_SINGULAR_COUPLING)


@pytest.mark.parametrize("N,L,m,r,ok", [
    (4096, 6, 64, 16, True),
    (4096, 6, 64, 65, False),     # r > 64
    (4100, 6, 64, 16, False),     # N != m 2^L
    (512, 1, 256, 16, True),
    (1024, 1, 512, 16, False),    # m > 256
    (64, 3, 8, 9, False),         # r > m
    (64, 0, 64, 1, False),        # L < 1
])
def test_descriptor_validation(hb, N, L, m, r, ok):
    d = hb.hodlr_desc(N=N, L=L, m=m, r=r, reserved=0, ldu=N, ldv=N)
    out = ctypes.c_size_t()
    code = hb._LIB.hodlr_factor_workspace_size(ctypes.byref(d), 0, ctypes.byref(out))
    assert (code == hb.HODLR_OK) == ok
    if ok:
        # the factor holds at least the leaf LUs and Y_big
        assert out.value >= 8 * (N * m + N * r * L)
    code = hb._LIB.hodlr_matvec_workspace_size(ctypes.byref(d), 3, ctypes.byref(out))
    assert (code == hb.HODLR_OK) == ok


def test_small_leading_dimension_rejected(hb):
    d = hb.hodlr_desc(N=256, L=2, m=64, r=4, reserved=0, ldu=255, ldv=256)
    out = ctypes.c_size_t()
    assert hb._LIB.hodlr_factor_workspace_size(ctypes.byref(d), 0, ctypes.byref(out)) == hb.HODLR_ERR_ARG


def test_bad_precision_rejected(hb):
    d = hb.hodlr_desc(N=256, L=2, m=64, r=4, reserved=0, ldu=256, ldv=256)
    out = ctypes.c_size_t()
    for bad in (-1, 4, 7):
        assert hb._LIB.hodlr_factor_workspace_size(ctypes.byref(d), bad, ctypes.byref(out)) == hb.HODLR_ERR_ARG
    for good in hb.PREC.values():
        assert hb._LIB.hodlr_factor_workspace_size(ctypes.byref(d), good, ctypes.byref(out)) == hb.HODLR_OK


def test_factor_rejects_small_workspace_before_any_launch(hb):
    d = hb.hodlr_desc(N=256, L=2, m=64, r=4, reserved=0, ldu=256, ldv=256)
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(1 << 20)   # never dereferenced: the size check fails first
    code = hb._LIB.hodlr_factor(ctypes.byref(d), fake, fake, fake, 0, fake, 16, None, ctypes.byref(h))
    assert code == hb.HODLR_ERR_WORKSPACE


@pytest.mark.parametrize("N,m,r,L", [(4096, 64, 16, 6), (1 << 18, 256, 64, 10), (1 << 20, 128, 32, 13)])
def test_product_costs_equal_oracle_loop_counts(N, m, r, L):
    from paper_2208_06290_gb300 import costs
    assert costs.factor_flops(N, m, r, L) == pytest.approx(ocosts.loop_factor_flops(N, m, r, L), rel=1e-12)
    for k in (1, 3):
        assert costs.solve_flops(N, m, r, L, k) == pytest.approx(ocosts.loop_solve_flops(N, m, r, L, k), rel=1e-12)
        assert costs.matvec_flops(N, m, r, L, k) == pytest.approx(ocosts.matvec_flops(N, m, r, L, k), rel=1e-12)


def test_binding_rejects_mismatched_widths_before_the_c_call(hb):
    """A Y narrower than X would let the kernels write past Y's end: the
    binding refuses it before any pointer reaches the library (CPU tensors
    suffice, the check comes first)."""
    N, L, r = 256, 2, 4
    D = torch.zeros(1 << L, N >> L, N >> L, dtype=torch.float64).transpose(1, 2)
    U = torch.zeros(r * L, N, dtype=torch.float64).T
    X = torch.zeros(3, N, dtype=torch.float64).T
    Y = torch.zeros(1, N, dtype=torch.float64).T
    for fn in (hb.hodlr_matvec_noalloc, hb.hodlr_matvec):
        with pytest.raises(ValueError, match="same number of columns"):
            fn(D, U, U, L, r, X, Y)


def test_binding_rejects_operands_off_the_current_device(hb):
    N, L, r = 256, 2, 4
    D = torch.zeros(1 << L, N >> L, N >> L, dtype=torch.float64).transpose(1, 2)
    U = torch.zeros(r * L, N, dtype=torch.float64).T
    X = torch.zeros(2, N, dtype=torch.float64).T
    with pytest.raises(ValueError, match="CUDA"):
        hb.hodlr_matvec_noalloc(D, U, U, L, r, X, X.clone())
    with pytest.raises(ValueError, match="CUDA"):
        hb._on_current_device(X)
