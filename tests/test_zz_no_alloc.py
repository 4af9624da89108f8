"""The allocation-free matvec, hodlr_matvec_noalloc, against hodlr_matvec.

It serves callers that cannot allocate device memory at the point of use
(inside a CUDA-graph capture, under a host application that owns all device
memory, in real-time loops): the library's fixed device scratch replaces the
caller's workspace. The test calls it through the C ABI twice in a row (the
scratch keeps the previous call's contents) and compares both results with
the workspace-based entry point, within the matvec tolerance used by the
other parity tests; it also checks that a problem too large for the fixed
scratch is refused before any work is enqueued. The file is named so that
pytest collects it last."""
import numpy as np
import pytest
import torch

from synth import HodlrShape, gaussian_rhs, synthetic_hodlr

pytestmark = pytest.mark.gpu


def _case(N, L, r, k, seed):
    D, U, V, g = synthetic_hodlr(HodlrShape(N, L, r), 4.0, seed)
    B = gaussian_rhs(N, k, g)
    return tuple(t.to("cuda") for t in (D, U, V, B))


@pytest.mark.parametrize("N,L,r,k", [(4096, 6, 16, 3), (1 << 14, 6, 32, 1), (2048, 3, 32, 2)])
def test_noalloc_matvec_matches_workspace_matvec(cuda_lib, N, L, r, k):
    hb = cuda_lib
    D, U, V, X = _case(N, L, r, k, seed=N + k)
    ref = hb.hodlr_matvec(D, U, V, L, r, X).cpu().numpy()
    for _ in range(2):
        Y = torch.full((k, N), float("nan"), dtype=torch.float64, device="cuda").T
        hb.hodlr_matvec_noalloc(D, U, V, L, r, X, Y)
        got = Y.cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-13


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
