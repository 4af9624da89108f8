"""The allocation-free matvec, hodlr_matvec_noalloc, against hodlr_matvec.

It serves callers that cannot allocate device memory at the point of use
(inside a CUDA-graph capture, under a host application that owns all device
memory, in real-time loops): the library's fixed device scratch replaces the
caller's workspace. The tests call it through the C ABI and compare with the
workspace-based entry point, element by element, within the matvec tolerance
used by the other parity tests:
* twice in a row on one problem with a call on another shape (other rank,
  other number of columns) in between, so that the second call finds the
  scratch full of unrelated partials: nothing in it may need to start at zero;
* one column where the four-launch one-column path's scratch is larger than
  the fixed array but the per-level partials fit, so that the general
  per-level path runs instead;
* a problem whose per-level partials exceed the array is refused before any
  work is enqueued.
The file is named so that pytest collects it last."""
import numpy as np
import pytest
import torch

from synth import HodlrShape, gaussian_rhs, synthetic_hodlr

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 32 << 20
MV_TOL = 1e-13


def _case(N, L, r, k, seed, device="cpu"):
    D, U, V, g = synthetic_hodlr(HodlrShape(N, L, r), 4.0, seed, device=device)
    B = gaussian_rhs(N, k, g, device=device)
    return tuple(t.to("cuda") for t in (D, U, V, B))


def _noalloc(hb, D, U, V, L, r, X):
    N, k = X.shape
    Y = torch.full((k, N), float("nan"), dtype=torch.float64, device="cuda").T
    hb.hodlr_matvec_noalloc(D, U, V, L, r, X, Y)
    return Y.cpu().numpy()


def _close(got, ref):
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < MV_TOL
    np.testing.assert_allclose(got, ref, rtol=0, atol=MV_TOL * np.abs(ref).max())


@pytest.mark.parametrize("N,L,r,k", [(4096, 6, 16, 3), (1 << 14, 6, 32, 1), (2048, 3, 32, 2)])
def test_noalloc_matvec_matches_workspace_matvec(cuda_lib, N, L, r, k):
    hb = cuda_lib
    D, U, V, X = _case(N, L, r, k, seed=N + k)
    ref = hb.hodlr_matvec(D, U, V, L, r, X).cpu().numpy()
    # another problem (other rank and width) that leaves its own partials in the scratch
    D2, U2, V2, X2 = _case(1 << 13, 5, 8 if r != 8 else 4, k + 2, seed=7 * N)
    r2 = U2.shape[1] // 5
    ref2 = hb.hodlr_matvec(D2, U2, V2, 5, r2, X2).cpu().numpy()
    _close(_noalloc(hb, D, U, V, L, r, X), ref)
    _close(_noalloc(hb, D2, U2, V2, 5, r2, X2), ref2)
    _close(_noalloc(hb, D, U, V, L, r, X), ref)


def test_noalloc_one_column_falls_back_to_the_general_path(cuda_lib):
    """2^13 leaves of 32 rows, rank 32, one column: the one-column path's
    scratch (per-leaf projections of every level, 2^13 * 32 * 13 doubles and
    more: 34 MiB) exceeds 32 MiB, the per-level partials (2^13 * 32 doubles)
    do not."""
    hb = cuda_lib
    N, L, r = 1 << 18, 13, 32
    desc = hb.hodlr_desc(N=N, L=L, m=N >> L, r=r, reserved=0, ldu=N, ldv=N)
    assert hb.hodlr_matvec_workspace_size(desc, 1) > SCRATCH_BYTES
    D, U, V, X = _case(N, L, r, 1, seed=5, device="cuda")
    ref = hb.hodlr_matvec(D, U, V, L, r, X).cpu().numpy()
    _close(_noalloc(hb, D, U, V, L, r, X), ref)
    _close(_noalloc(hb, D, U, V, L, r, X), ref)


def test_noalloc_matvec_rejects_problems_beyond_its_scratch(cuda_lib):
    hb = cuda_lib
    # 2^13 leaves of 16 rows, rank 16, 40 columns: the per-node partials need
    # 2^13 * 16 * 40 doubles = 40 MiB > 32 MiB
    N, L, r, k = 1 << 17, 13, 16, 40
    D, U, V, X = _case(N, L, r, k, seed=1)
    Y = torch.empty(k, N, dtype=torch.float64, device="cuda").T
    with pytest.raises(hb.HodlrError) as ei:
        hb.hodlr_matvec_noalloc(D, U, V, L, r, X, Y)
    assert ei.value.code == hb.HODLR_ERR_SCRATCH_LIMIT
