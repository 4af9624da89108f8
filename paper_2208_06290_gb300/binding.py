"""Thin ctypes binding of libhodlr (include/hodlr.h).

Each ``hodlr_*`` function here has the name of the C entry point it wraps and
only marshals arguments: it checks torch tensors (device, dtype, column-major
layout), allocates the caller-owned workspace as a torch uint8 tensor, passes
raw device pointers and the current CUDA stream, and turns a status code into
an exception. All arithmetic runs in the library's CUDA kernels. There is no
CPU fallback: if the library cannot be loaded, importing this module raises.

Tensor layouts (as in the C ABI; see ``synth.generators`` for generators):
* D: (2^L, m, m) float64 CUDA tensor with column-major blocks, strides (m*m, 1, m);
* U, V: (N, r*L) float64 CUDA, column-major (stride (1, ld), ld >= N);
* B, X, Y: (N, k) float64 CUDA, column-major.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

HODLR_OK = 0
HODLR_ERR_ARG = 1
HODLR_ERR_WORKSPACE = 2
HODLR_ERR_CUDA = 3
HODLR_ERR_SINGULAR_LEAF = 4
HODLR_ERR_SINGULAR_COUPLING = 5
HODLR_ERR_NONFINITE = 6
HODLR_ERR_NOT_CONVERGED = 7
HODLR_ERR_TIMEOUT = 8
HODLR_ERR_SCRATCH_LIMIT = 9

PREC = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3}

EXPORTED = (
    "hodlr_strerror", "hodlr_factor_workspace_size", "hodlr_factor", "hodlr_factor_status", "hodlr_free",
    "hodlr_solve_workspace_size", "hodlr_solve", "hodlr_solve_adjoint", "hodlr_logdet",
    "hodlr_matvec_workspace_size", "hodlr_matvec", "hodlr_refine_workspace_size", "hodlr_solve_refined",
    "hodlr_gmres", "hodlr_launch_count", "hodlr_profile_enable", "hodlr_profile_reset", "hodlr_profile_read",
    "hodlr_profile_name", "hodlr_profile_work", "hodlr_tc_enable", "hodlr_grad_workspace_size", "hodlr_grad",
    "hodlr_matvec_noalloc", "hodlr_probe_fp64_fma", "hodlr_coupling_fp64_enable",
    "hodlr_compress_workspace_size", "hodlr_compress", "hodlr_factor_inplace_workspace_size",
    "hodlr_factor_inplace", "hodlr_pack_level_ranks",
)

KERNEL = {"bie_star": 0, "gaussian": 1, "matern32": 2}


class hodlr_kernel_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("dim", ctypes.c_int32), ("points", ctypes.c_void_p),
                ("scale", ctypes.c_double), ("nugget", ctypes.c_double), ("tol", ctypes.c_double)]


class HodlrError(RuntimeError):
    def __init__(self, code, where=None, detail=None, msg=""):
        self.code, self.where, self.detail = code, where, detail
        super().__init__(f"{msg}{_strerror(code)} (status {code}, where={where}, detail={detail})")


class hodlr_desc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("L", ctypes.c_int32), ("m", ctypes.c_int32), ("r", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("ldu", ctypes.c_int64), ("ldv", ctypes.c_int64)]


_c = ctypes
_vp, _i32, _i64, _sz, _dbl = _c.c_void_p, _c.c_int32, _c.c_int64, _c.c_size_t, _c.c_double
_SIGS = {
    "hodlr_strerror": ([_c.c_int], _c.c_char_p),
    "hodlr_factor_workspace_size": ([_vp, _c.c_int, _c.POINTER(_sz)], _c.c_int),
    "hodlr_factor": ([_vp, _vp, _vp, _vp, _c.c_int, _vp, _sz, _vp, _c.POINTER(_vp)], _c.c_int),
    "hodlr_factor_status": ([_vp, _c.POINTER(_i64), _c.POINTER(_i64)], _c.c_int),
    "hodlr_free": ([_vp], None),
    "hodlr_solve_workspace_size": ([_vp, _i32, _c.POINTER(_sz)], _c.c_int),
    "hodlr_solve": ([_vp, _vp, _i64, _i32, _vp, _sz, _vp], _c.c_int),
    "hodlr_solve_adjoint": ([_vp, _vp, _i64, _i32, _vp, _sz, _vp], _c.c_int),
    "hodlr_logdet": ([_vp, _vp, _c.POINTER(_dbl), _c.POINTER(_dbl)], _c.c_int),
    "hodlr_matvec_workspace_size": ([_vp, _i32, _c.POINTER(_sz)], _c.c_int),
    "hodlr_matvec": ([_vp, _vp, _vp, _vp, _vp, _i64, _vp, _i64, _i32, _vp, _sz, _vp], _c.c_int),
    "hodlr_refine_workspace_size": ([_vp, _i32, _i32, _c.POINTER(_sz)], _c.c_int),
    "hodlr_solve_refined": ([_vp, _vp, _vp, _vp, _vp, _i64, _vp, _i64, _i32, _dbl, _i32, _i32, _i32, _vp, _sz,
                             _vp, _c.POINTER(_i32), _c.POINTER(_dbl)], _c.c_int),
    "hodlr_gmres": ([_vp, _vp, _vp, _vp, _vp, _i64, _vp, _i64, _i32, _dbl, _i32, _i32, _vp, _sz, _vp,
                     _c.POINTER(_i32), _c.POINTER(_dbl)], _c.c_int),
    "hodlr_launch_count": ([], _i64),
    "hodlr_profile_enable": ([_i32], None),
    "hodlr_profile_reset": ([], None),
    "hodlr_profile_read": ([_c.POINTER(_dbl), _c.POINTER(_i64), _i32], _i32),
    "hodlr_profile_name": ([_i32], _c.c_char_p),
    "hodlr_profile_work": ([_c.POINTER(_dbl), _c.POINTER(_dbl), _i32], _i32),
    "hodlr_tc_enable": ([_i32], None),
    "hodlr_coupling_fp64_enable": ([_i32], None),
    "hodlr_compress_workspace_size": ([_vp, _c.POINTER(_sz)], _c.c_int),
    "hodlr_compress": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp], _c.c_int),
    "hodlr_factor_inplace_workspace_size": ([_vp, _c.POINTER(_sz)], _c.c_int),
    "hodlr_pack_level_ranks": ([_vp, _c.POINTER(_i32), _vp, _i64, _vp, _i64, _vp, _vp, _vp, _sz, _vp], _c.c_int),
    "hodlr_factor_inplace": ([_vp, _vp, _vp, _vp, _vp, _sz, _vp, _c.POINTER(_vp)], _c.c_int),
    "hodlr_matvec_noalloc": ([_vp, _vp, _vp, _vp, _vp, _i64, _vp, _i64, _i32, _vp], _c.c_int),
    "hodlr_probe_fp64_fma": ([_i64, _i32, _vp, _vp, _c.POINTER(_i64)], _c.c_int),
    "hodlr_grad_workspace_size": ([_vp, _i32, _c.POINTER(_sz)], _c.c_int),
    "hodlr_grad": ([_vp, _vp, _vp, _vp, _i64, _i32, _vp, _vp, _vp, _vp, _i64, _vp, _sz, _vp, _c.POINTER(_dbl)],
                   _c.c_int),
}


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Build (if needed) and load libhodlr.so; raises if that is impossible."""
    path = path or _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libhodlr not found at {path}")
    lib = ctypes.CDLL(path)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_LIB = load_library()


def _strerror(code) -> str:
    return _LIB.hodlr_strerror(int(code)).decode()


def _check(code, msg=""):
    if code != HODLR_OK:
        raise HodlrError(code, msg=msg)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ld(t: torch.Tensor, N: int) -> int:
    if t.dim() != 2 or t.shape[0] != N:
        raise ValueError(f"expected an (N={N}, k) matrix, got {tuple(t.shape)}")
    if not t.is_cuda or t.dtype != torch.float64:
        raise ValueError("expected a float64 CUDA tensor")
    if t.stride(0) != 1:
        raise ValueError("expected a column-major matrix (stride (1, ld))")
    return t.stride(1) if t.shape[1] > 1 else max(N, t.stride(1))


def _on_current_device(*ts: torch.Tensor) -> None:
    """Every operand must live on the current CUDA device: the library
    launches on that device's current stream (and the allocation-free matvec
    takes that device's scratch)."""
    for t in ts:
        if t is None:
            continue
        if not t.is_cuda or t.device.index != torch.cuda.current_device():
            raise ValueError(f"operand on {t.device}, expected the current CUDA device "
                             "(use torch.cuda.device(...) around the call)")


def _same_width(X: torch.Tensor, Y: torch.Tensor) -> None:
    if X.dim() != 2 or Y.dim() != 2 or Y.shape[1] != X.shape[1]:
        raise ValueError(f"X and Y must have the same number of columns, got {tuple(X.shape)} and {tuple(Y.shape)}")


def make_desc(N: int, L: int, r: int, U: torch.Tensor | None = None, V: torch.Tensor | None = None) -> hodlr_desc:
    ldu = _ld(U, N) if U is not None else N
    ldv = _ld(V, N) if V is not None else N
    return hodlr_desc(N=N, L=L, m=N >> L, r=r, reserved=0, ldu=ldu, ldv=ldv)


def _check_D(D: torch.Tensor, N: int, L: int):
    m = N >> L
    if tuple(D.shape) != (1 << L, m, m) or D.stride() != (m * m, 1, m):
        raise ValueError("D must be (2^L, m, m) with column-major blocks, strides (m*m, 1, m)")
    if not D.is_cuda or D.dtype != torch.float64:
        raise ValueError("D must be a float64 CUDA tensor")


def _ptr(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


class FactorHandle:
    """A factor made by ``hodlr_factor``: the C handle plus the torch tensors
    it points into (its workspace, and V in FP64), kept alive with it."""

    def __init__(self, handle, desc, prec, workspace, keep):
        self.handle, self.desc, self.prec = handle, desc, prec
        self.workspace, self._keep = workspace, keep

    @property
    def N(self):
        return self.desc.N

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _LIB is not None:
            _LIB.hodlr_free(h)


# ----------------------------------------------------------------- entry points
def hodlr_factor_workspace_size(desc: hodlr_desc, prec: str = "fp64") -> int:
    out = ctypes.c_size_t()
    _check(_LIB.hodlr_factor_workspace_size(ctypes.byref(desc), PREC[prec], ctypes.byref(out)))
    return out.value


def hodlr_factor(D, U, V, L: int, r: int, prec: str = "fp64") -> FactorHandle:
    N = U.shape[0]
    _check_D(D, N, L)
    _on_current_device(D, U, V)
    desc = make_desc(N, L, r, U, V)
    if U.shape[1] != r * L or V.shape[1] != r * L:
        raise ValueError("U, V must have r*L columns")
    ws = _workspace(hodlr_factor_workspace_size(desc, prec), U.device)
    h = ctypes.c_void_p()
    _check(_LIB.hodlr_factor(ctypes.byref(desc), _ptr(D), _ptr(U), _ptr(V), PREC[prec], _ptr(ws), ws.numel(),
                             _stream(), ctypes.byref(h)), "hodlr_factor: ")
    return FactorHandle(h, desc, prec, ws, (V,) if prec == "fp64" else ())


def hodlr_factor_inplace(D, U, V, L: int, r: int) -> FactorHandle:
    """FP64 factorization that overwrites D with the leaf LUs and U (leading
    dimension N) with Y_big; the returned factor keeps D, U and V alive."""
    N = U.shape[0]
    _check_D(D, N, L)
    _on_current_device(D, U, V)
    desc = make_desc(N, L, r, U, V)
    if desc.ldu != N or U.shape[1] != r * L or V.shape[1] != r * L:
        raise ValueError("U must be (N, r L) with leading dimension N; V (N, r L)")
    out = ctypes.c_size_t()
    _check(_LIB.hodlr_factor_inplace_workspace_size(ctypes.byref(desc), ctypes.byref(out)))
    ws = _workspace(out.value, U.device)
    h = ctypes.c_void_p()
    _check(_LIB.hodlr_factor_inplace(ctypes.byref(desc), _ptr(D), _ptr(U), _ptr(V), _ptr(ws), ws.numel(), _stream(),
                                     ctypes.byref(h)), "hodlr_factor_inplace: ")
    return FactorHandle(h, desc, "fp64", ws, (D, U, V))


def hodlr_factor_status(F: FactorHandle):
    where, detail = ctypes.c_int64(), ctypes.c_int64()
    code = _LIB.hodlr_factor_status(F.handle, ctypes.byref(where), ctypes.byref(detail))
    return code, where.value, detail.value


def hodlr_solve_workspace_size(F: FactorHandle, k: int) -> int:
    out = ctypes.c_size_t()
    _check(_LIB.hodlr_solve_workspace_size(F.handle, k, ctypes.byref(out)))
    return out.value


def _solve(fn, F: FactorHandle, B: torch.Tensor):
    ldb = _ld(B, F.N)
    _on_current_device(B, F.workspace)
    k = B.shape[1]
    ws = _workspace(hodlr_solve_workspace_size(F, k), B.device)
    _check(fn(F.handle, _ptr(B), ldb, k, _ptr(ws), ws.numel(), _stream()))
    return B


def hodlr_solve(F: FactorHandle, B: torch.Tensor) -> torch.Tensor:
    """B <- A^{-1} B in place (returns B)."""
    return _solve(_LIB.hodlr_solve, F, B)


def hodlr_solve_adjoint(F: FactorHandle, B: torch.Tensor) -> torch.Tensor:
    """B <- A^{-T} B in place (returns B)."""
    return _solve(_LIB.hodlr_solve_adjoint, F, B)


def hodlr_logdet(F: FactorHandle):
    """(sign, log|det A|); raises on a device-side factor error."""
    sign, la = ctypes.c_double(), ctypes.c_double()
    code = _LIB.hodlr_logdet(F.handle, _stream(), ctypes.byref(sign), ctypes.byref(la))
    if code != HODLR_OK:
        c, w, d = hodlr_factor_status(F)
        raise HodlrError(code, w, d, "hodlr_logdet: ")
    return sign.value, la.value


def hodlr_matvec_workspace_size(desc: hodlr_desc, k: int) -> int:
    out = ctypes.c_size_t()
    _check(_LIB.hodlr_matvec_workspace_size(ctypes.byref(desc), k, ctypes.byref(out)))
    return out.value


def hodlr_matvec(D, U, V, L: int, r: int, X: torch.Tensor, Y: torch.Tensor | None = None) -> torch.Tensor:
    """Y = A X in FP64."""
    N = U.shape[0]
    if Y is not None:
        _same_width(X, Y)
    _check_D(D, N, L)
    desc = make_desc(N, L, r, U, V)
    ldx = _ld(X, N)
    k = X.shape[1]
    if Y is None:
        Y = torch.empty(k, N, dtype=torch.float64, device=X.device).T
    ldy = _ld(Y, N)
    _on_current_device(D, U, V, X, Y)
    ws = _workspace(hodlr_matvec_workspace_size(desc, k), X.device)
    _check(_LIB.hodlr_matvec(ctypes.byref(desc), _ptr(D), _ptr(U), _ptr(V), _ptr(X), ldx, _ptr(Y), ldy, k,
                             _ptr(ws), ws.numel(), _stream()), "hodlr_matvec: ")
    return Y


def hodlr_refine_workspace_size(F: FactorHandle, k: int, restart: int = 0) -> int:
    out = ctypes.c_size_t()
    _check(_LIB.hodlr_refine_workspace_size(F.handle, k, restart, ctypes.byref(out)))
    return out.value


def hodlr_solve_refined(F: FactorHandle, D, U, V, B, tol=1e-10, max_iter=50, X=None, raise_on_fail=True,
                        restart=0, gmres_max_iter=300):
    """Iterative refinement with FP64 residuals, continued by FGMRES(restart)
    when it stalls (restart > 0); returns (X, iters, relres, status)."""
    N = F.N
    ldb = _ld(B, N)
    k = B.shape[1]
    if X is not None:
        _same_width(B, X)
    if X is None:
        X = torch.empty(k, N, dtype=torch.float64, device=B.device).T
    ldx = _ld(X, N)
    _check_D(D, N, F.desc.L)
    _on_current_device(D, U, V, B, X, F.workspace)
    ws = _workspace(hodlr_refine_workspace_size(F, k, restart), B.device)
    it, rr = ctypes.c_int32(), ctypes.c_double()
    code = _LIB.hodlr_solve_refined(F.handle, _ptr(D), _ptr(U), _ptr(V), _ptr(B), ldb, _ptr(X), ldx, k, tol,
                                    max_iter, restart, gmres_max_iter if restart > 0 else 0, _ptr(ws), ws.numel(),
                                    _stream(), ctypes.byref(it), ctypes.byref(rr))
    if raise_on_fail and code != HODLR_OK:
        raise HodlrError(code, msg=f"hodlr_solve_refined (iters={it.value}, relres={rr.value:.3e}): ")
    return X, it.value, rr.value, code


def hodlr_gmres(F: FactorHandle, D, U, V, B, tol=1e-10, restart=30, max_iter=300, X=None, raise_on_fail=True):
    """Flexible GMRES right-preconditioned by F; returns (X, iters, relres, status)."""
    N = F.N
    ldb = _ld(B, N)
    k = B.shape[1]
    if X is not None:
        _same_width(B, X)
    if X is None:
        X = torch.empty(k, N, dtype=torch.float64, device=B.device).T
    ldx = _ld(X, N)
    _check_D(D, N, F.desc.L)
    _on_current_device(D, U, V, B, X, F.workspace)
    ws = _workspace(hodlr_refine_workspace_size(F, k, restart), B.device)
    it, rr = ctypes.c_int32(), ctypes.c_double()
    code = _LIB.hodlr_gmres(F.handle, _ptr(D), _ptr(U), _ptr(V), _ptr(B), ldb, _ptr(X), ldx, k, tol, restart,
                            max_iter, _ptr(ws), ws.numel(), _stream(), ctypes.byref(it), ctypes.byref(rr))
    if raise_on_fail and code != HODLR_OK:
        raise HodlrError(code, msg=f"hodlr_gmres (iters={it.value}, relres={rr.value:.3e}): ")
    return X, it.value, rr.value, code


# ------------------------------------------------------------------ diagnostics
def hodlr_launch_count() -> int:
    return int(_LIB.hodlr_launch_count())


def hodlr_profile_enable(on: bool = True) -> None:
    _LIB.hodlr_profile_enable(1 if on else 0)


def hodlr_profile_reset() -> None:
    _LIB.hodlr_profile_reset()


def hodlr_profile_read() -> dict:
    """{kernel class: (milliseconds, launches)}; synchronizes the device."""
    n = 16
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int64 * n)()
    k = _LIB.hodlr_profile_read(ms, cnt, n)
    return {hodlr_profile_name(i): (ms[i], cnt[i]) for i in range(min(k, n))}


def hodlr_profile_work() -> dict:
    """{kernel class: (algorithmic bytes, algorithmic flops)} of the profiled launches."""
    n = 16
    by = (ctypes.c_double * n)()
    fl = (ctypes.c_double * n)()
    k = _LIB.hodlr_profile_work(by, fl, n)
    return {hodlr_profile_name(i): (by[i], fl[i]) for i in range(min(k, n))}


def hodlr_profile_name(i: int) -> str:
    return _LIB.hodlr_profile_name(i).decode()


def hodlr_probe_fp64_fma(iters: int, blocks_per_sm: int, out: torch.Tensor) -> int:
    """Enqueue the FP64 FMA probe on the current stream; returns its FMA count
    (time it with CUDA events on that stream)."""
    _on_current_device(out)
    n = ctypes.c_int64()
    _check(_LIB.hodlr_probe_fp64_fma(int(iters), int(blocks_per_sm), _ptr(out), _stream(), ctypes.byref(n)))
    return n.value


def hodlr_coupling_fp64_enable(on: bool = True) -> None:
    """BF16 factor: coupling products in FP64 (on) or FP32 (off, default)."""
    _LIB.hodlr_coupling_fp64_enable(1 if on else 0)


def hodlr_tc_enable(on: bool = True) -> None:
    """Select tensor-core (on, default) or CUDA-core kernels for the BF16 factor."""
    _LIB.hodlr_tc_enable(1 if on else 0)


# ------------------------------------------------------------------- gradient
def hodlr_grad_workspace_size(F: FactorHandle, k: int) -> int:
    out = ctypes.c_size_t()
    _check(_LIB.hodlr_grad_workspace_size(F.handle, k, ctypes.byref(out)))
    return out.value


def hodlr_grad(F: FactorHandle, U, V, B, want_loss: bool = True):
    """(loss, dD, dU, dV, dB) of loss = sum_j b_j^T A^{-1} b_j + log|det A| for
    the FP64 factor F of (D, U, V); dD in D's layout, dU / dV / dB column-major."""
    N = F.N
    ldb = _ld(B, N)
    k = B.shape[1]
    m, L = F.desc.m, F.desc.L
    rL = F.desc.r * L
    dev = B.device
    _on_current_device(U, V, B, F.workspace)
    dD = torch.empty(1 << L, m, m, dtype=torch.float64, device=dev).transpose(1, 2)
    dU = torch.empty(rL, N, dtype=torch.float64, device=dev).T
    dV = torch.empty(rL, N, dtype=torch.float64, device=dev).T
    dB = torch.empty(k, N, dtype=torch.float64, device=dev).T
    ws = _workspace(hodlr_grad_workspace_size(F, k), dev)
    loss = ctypes.c_double()
    _check(_LIB.hodlr_grad(F.handle, _ptr(U), _ptr(V), _ptr(B), ldb, k, _ptr(dD), _ptr(dU), _ptr(dV), _ptr(dB), N,
                           _ptr(ws), ws.numel(), _stream(), ctypes.byref(loss) if want_loss else None),
           "hodlr_grad: ")
    return (loss.value if want_loss else None), dD, dU, dV, dB


def hodlr_matvec_noalloc(D, U, V, L: int, r: int, X: torch.Tensor, Y: torch.Tensor) -> torch.Tensor:
    """Y = A X in FP64 without any allocation by the library or this wrapper:
    the library's fixed device scratch replaces the workspace. Y must be
    preallocated (column-major)."""
    N = U.shape[0]
    _same_width(X, Y)
    _check_D(D, N, L)
    desc = make_desc(N, L, r, U, V)
    ldx, ldy = _ld(X, N), _ld(Y, N)
    _on_current_device(D, U, V, X, Y)
    _check(_LIB.hodlr_matvec_noalloc(ctypes.byref(desc), _ptr(D), _ptr(U), _ptr(V), _ptr(X), ldx, _ptr(Y), ldy,
                                     X.shape[1], _stream()), "hodlr_matvec_noalloc: ")
    return Y


# --------------------------------------------------------------- construction
def hodlr_compress(N: int, L: int, r: int, kind: str, points: torch.Tensor | None = None, scale: float = 1.0,
                   nugget: float = 0.0, want_pivots: bool = False, device=None, tol: float = 0.0,
                   want_ranks: bool = False):
    """(D, U, V[, pivots][, ranks]) of the HODLR approximation of a built-in
    kernel or BIE matrix, built on the GPU (leaf blocks exact, off-diagonal
    blocks by a partial-pivoted cross approximation at rank r, or stopped at
    the relative pivot tolerance tol: per-block ranks, zero-padded bases).
    points: (N, dim) float64 CUDA tensor in tree order (kernel matrices),
    None for 'bie_star'."""
    if kind not in KERNEL:
        raise ValueError(f"kind must be one of {sorted(KERNEL)}")
    m = N >> L
    if device is None:
        device = points.device if points is not None else torch.device("cuda", torch.cuda.current_device())
    dim = 0
    if points is not None:
        if points.dim() != 2 or points.shape[0] != N or not points.is_contiguous() or points.dtype != torch.float64:
            raise ValueError("points must be a contiguous (N, dim) float64 tensor")
        _on_current_device(points)
        dim = points.shape[1]
    elif kind != "bie_star":
        raise ValueError("kernel matrices need points")
    desc = hodlr_desc(N=N, L=L, m=m, r=r, reserved=0, ldu=N, ldv=N)
    kd = hodlr_kernel_desc(kind=KERNEL[kind], dim=dim, points=points.data_ptr() if points is not None else None,
                           scale=float(scale), nugget=float(nugget), tol=float(tol))
    D = torch.empty(1 << L, m, m, dtype=torch.float64, device=device).transpose(1, 2)
    U = torch.empty(r * L, N, dtype=torch.float64, device=device).T
    V = torch.empty(r * L, N, dtype=torch.float64, device=device).T
    piv = torch.empty(2 * r * ((2 << L) - 2), dtype=torch.int32, device=device) if want_pivots else None
    rk = torch.empty((2 << L) - 2, dtype=torch.int32, device=device) if want_ranks else None
    out = ctypes.c_size_t()
    _check(_LIB.hodlr_compress_workspace_size(ctypes.byref(desc), ctypes.byref(out)))
    ws = _workspace(out.value, device)
    _check(_LIB.hodlr_compress(ctypes.byref(desc), ctypes.byref(kd), _ptr(D), _ptr(U), _ptr(V),
                               _ptr(piv) if piv is not None else None, _ptr(rk) if rk is not None else None,
                               _ptr(ws), ws.numel(), _stream()), "hodlr_compress: ")
    return (D, U, V) + ((piv,) if want_pivots else ()) + ((rk,) if want_ranks else ())


def hodlr_pack_level_ranks(Ur: torch.Tensor, Vr: torch.Tensor, L: int, level_ranks, r: int | None = None):
    """Uniform (U, V) of width r (default max rank) from the ragged per-level
    layout (level c's bases in columns sum(r_1..r_{c-1}) .. + r_c - 1)."""
    lr = [int(x) for x in level_ranks]
    if len(lr) != L:
        raise ValueError("level_ranks needs L entries")
    r = max(lr) if r is None else r
    N = Ur.shape[0]
    ldur, ldvr = _ld(Ur, N), _ld(Vr, N)
    if Ur.shape[1] != sum(lr) or Vr.shape[1] != sum(lr):
        raise ValueError("Ur, Vr must have sum(level_ranks) columns")
    _on_current_device(Ur, Vr)
    U = torch.empty(r * L, N, dtype=torch.float64, device=Ur.device).T
    V = torch.empty(r * L, N, dtype=torch.float64, device=Ur.device).T
    desc = hodlr_desc(N=N, L=L, m=N >> L, r=r, reserved=0, ldu=N, ldv=N)
    ws = _workspace(2 * L * 4, Ur.device)
    arr = (ctypes.c_int32 * L)(*lr)
    _check(_LIB.hodlr_pack_level_ranks(ctypes.byref(desc), arr, _ptr(Ur), ldur, _ptr(Vr), ldvr, _ptr(U), _ptr(V),
                                       _ptr(ws), ws.numel(), _stream()), "hodlr_pack_level_ranks: ")
    return U, V
