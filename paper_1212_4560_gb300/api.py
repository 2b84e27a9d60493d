"""Thin binding of the libgenp C ABI: the same entry points, taking torch
CUDA tensors (PyTorch supplies device memory and streams only; every step
of the method runs in the library's kernels).

Names follow include/genp.h without the ``genp_`` prefix.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import torch

from . import _lib
from ._lib import BF16, BF16_SLICED, BF16X3, CIRCULANT, FP8_E4M3, FP32, FP64, GAUSSIAN, SPARSE_PM1, GenpError, check

_PREC_OF_DTYPE = {torch.float64: FP64, torch.float32: FP32}


def _stream(stream=None) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libgenp takes CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def _ld(t: torch.Tensor) -> int:
    """Leading dimension of a row-major 2-D view (unit column stride required)."""
    if t.dim() != 2 or (t.stride(1) != 1 and t.size(1) > 1):
        raise ValueError("expected a row-major 2-D tensor with unit column stride")
    return max(t.stride(0), t.size(1), 1)


def version() -> str:
    return _lib.load().genp_version().decode()


def status_string(status: int) -> str:
    return _lib.load().genp_status_string(status).decode()


class Multiplier:
    """Owns a genp_multiplier handle."""

    def __init__(self, handle, n, kind, nnz):
        self.handle, self.n, self.kind, self.nnz = handle, n, kind, nnz

    def __del__(self):
        if getattr(self, "handle", None):
            _lib.load().genp_multiplier_destroy(self.handle)
            self.handle = None


class Factors:
    """Owns a genp_factors handle (and keeps the factored tensor alive)."""

    def __init__(self, handle, C, prec):
        self.handle, self.C, self.prec = handle, C, prec

    @property
    def n(self):
        return self.C.size(0)

    def __del__(self):
        if getattr(self, "handle", None):
            _lib.load().genp_factors_destroy(self.handle)
            self.handle = None


def make_multiplier(kind: int, n: int, seed: int, stream_id: int = 0, scale: float | None = None,
                    nnz_per_col: int = 4, value_grid: int = FP64, stream=None, side: int = 0) -> Multiplier:
    """genp_make_multiplier (and genp_multiplier_side for side = LEFT).
    Default scale: 1/sqrt(n) (Gaussian, variance 1/n) and 1 (circulant,
    Toeplitz)."""
    if scale is None:
        scale = 1.0 / math.sqrt(n) if kind == GAUSSIAN else 1.0
    h = ctypes.c_void_p()
    check(_lib.load().genp_make_multiplier(kind, n, seed, stream_id, float(scale), nnz_per_col, value_grid,
                                           _stream(stream), ctypes.byref(h)), "genp_make_multiplier")
    G = Multiplier(h, n, kind, nnz_per_col if kind == SPARSE_PM1 else 0)
    if side:
        prev = _lib.load().genp_multiplier_side(h, side)
        if prev < 0:
            check(prev, "genp_multiplier_side")
    return G


def redraw_multiplier(G: Multiplier, seed: int, stream_id: int = 0, stream=None) -> None:
    """genp_redraw_multiplier: new random G in the same storage (no allocation)."""
    check(_lib.load().genp_redraw_multiplier(G.handle, seed, stream_id, _stream(stream)), "genp_redraw_multiplier")


def launch_count() -> int:
    """genp_launch_count: kernels launched by the library so far."""
    return int(_lib.load().genp_launch_count())


def multiplier_export(G: Multiplier, dense=None, first_col=None, rows=None, signs=None, stream=None) -> None:
    check(_lib.load().genp_multiplier_export(G.handle, _ptr(dense), _ld(dense) if dense is not None else 0,
                                             _ptr(first_col), _ptr(rows), _ptr(signs), _stream(stream)),
          "genp_multiplier_export")


def precondition(G: Multiplier, A: torch.Tensor, C: torch.Tensor, c_prec: int | None = None, stream=None) -> None:
    """genp_precondition: C = A G."""
    a_prec = _PREC_OF_DTYPE[A.dtype]
    if c_prec is None:
        c_prec = _PREC_OF_DTYPE[C.dtype]
    check(_lib.load().genp_precondition(G.handle, _ptr(A), _ld(A), a_prec, _ptr(C), _ld(C), c_prec,
                                        _stream(stream)), "genp_precondition")


def factor(C: torch.Tensor, prec: int | None = None, nb: int = 0, stream=None) -> Factors:
    """genp_factor: in-place GENP of C."""
    if prec is None:
        prec = _PREC_OF_DTYPE[C.dtype]
    h = ctypes.c_void_p()
    check(_lib.load().genp_factor(_ptr(C), C.size(0), _ld(C), prec, nb, _stream(stream), ctypes.byref(h)),
          "genp_factor")
    return Factors(h, C, prec)


def block_factor(C: torch.Tensor, nb: int = 64, stream=None) -> Factors:
    """genp_block_factor: in-place block Gaussian elimination of the FP64
    matrix C with explicit inverses of its nb x nb pivot blocks."""
    if C.dtype != torch.float64:
        raise ValueError("block GE takes an FP64 matrix")
    h = ctypes.c_void_p()
    check(_lib.load().genp_block_factor(_ptr(C), C.size(0), _ld(C), nb, _stream(stream), ctypes.byref(h)),
          "genp_block_factor")
    return Factors(h, C, FP64)


def refactor(F: Factors, C: torch.Tensor, stream=None) -> None:
    check(_lib.load().genp_refactor(F.handle, _ptr(C), _ld(C), _stream(stream)), "genp_refactor")
    F.C = C


def solve(F: Factors, G: Multiplier, B: torch.Tensor, X: torch.Tensor, stream=None) -> None:
    """genp_solve: X = G U^-1 L^-1 B (B, X float64, n x nrhs)."""
    check(_lib.load().genp_solve(F.handle, G.handle, _ptr(B), _ld(B), B.size(1), _ptr(X), _ld(X), _stream(stream)),
          "genp_solve")


def refine(A: torch.Tensor, F: Factors, G: Multiplier, B: torch.Tensor, X: torch.Tensor, tol: float = 1e-15,
           max_iter: int = 10, method: int = 0, stream=None) -> None:
    """genp_refine: FP64 iterative refinement of X in place."""
    check(_lib.load().genp_refine(_ptr(A), _ld(A), F.handle, G.handle, _ptr(B), _ld(B), B.size(1), _ptr(X), _ld(X),
                                  float(tol), int(max_iter), int(method), _stream(stream)), "genp_refine")


def adjoint(F: Factors, G: Multiplier, gX: torch.Tensor, X: torch.Tensor | None, dA: torch.Tensor | None,
            dB: torch.Tensor | None, stream=None) -> None:
    """genp_adjoint: Lambda = L^-T U^-T G^T gX, dA = -Lambda X^T, dB = Lambda."""
    check(_lib.load().genp_adjoint(F.handle, G.handle, _ptr(gX), _ld(gX), _ptr(X), _ld(X) if X is not None else 0,
                                   gX.size(1), _ptr(dA), _ld(dA) if dA is not None else 0, _ptr(dB),
                                   _ld(dB) if dB is not None else 0, _stream(stream)), "genp_adjoint")


@dataclass
class Info:
    status: int
    refine_iters: int
    breakdown_step: int
    min_abs_pivot: float
    max_abs_pivot: float
    growth: float
    bwd_err: list
    krylov_steps: int = 0


def info_fetch(F: Factors, stream=None) -> Info:
    """genp_info_fetch (synchronizes the stream)."""
    out = _lib.GenpInfo()
    check(_lib.load().genp_info_fetch(F.handle, ctypes.byref(out), _stream(stream)), "genp_info_fetch")
    errs = [e for e in out.bwd_err[: out.refine_iters + 1] if e >= 0]
    return Info(out.status, out.refine_iters, out.breakdown_step, out.min_abs_pivot, out.max_abs_pivot, out.growth,
                errs, out.krylov_steps)


def solve_system(A: torch.Tensor, B: torch.Tensor, kind: int = GAUSSIAN, seed: int = 0, prec: int = FP64,
                 refine_steps: int = 10, tol: float = 1e-15, nb: int = 0, method: int = 0, stream=None,
                 side: int = 0):
    """The whole method on one system: G, C = A G, GENP(C), X = G U^-1 L^-1 B,
    FP64 refinement (method 0 classic, 1 GMRES-IR); side = LEFT: C = G A,
    X = U^-1 L^-1 G B.  Returns (X, info, G, F)."""
    n = A.size(0)
    f64 = prec in (FP64, BF16_SLICED)
    # FP32-grid draws for the FP32 factorization, BF16 / FP8 grids for the
    # tensor-core ones, and the sliced product's fixed-point grid for the
    # sliced one (one digit by default: A G then forms nd digit products
    # instead of nd (nd + 1) / 2)
    grid = {FP64: FP64, BF16: BF16, BF16X3: BF16, FP8_E4M3: FP8_E4M3, BF16_SLICED: BF16_SLICED}.get(prec, FP32)
    G = make_multiplier(kind, n, seed, value_grid=grid, stream=stream, side=side)
    C = torch.empty((n, n), dtype=torch.float64 if f64 else torch.float32, device=A.device)
    A64 = A if A.dtype == torch.float64 else A.double()
    precondition(G, A64 if f64 else A, C, c_prec=prec, stream=stream)
    F = factor(C, prec=prec, nb=nb, stream=stream)
    B64 = B.double().contiguous()
    X = torch.empty_like(B64)
    solve(F, G, B64, X, stream=stream)
    if refine_steps > 0:
        refine(A64, F, G, B64, X, tol=tol, max_iter=refine_steps, method=method, stream=stream)
    return X, info_fetch(F, stream=stream), G, F


def lowrank(A: torch.Tensor, r: int, kind: int = GAUSSIAN, seed: int = 0, stream_id: int = 0, stream=None):
    """genp_lowrank: the sketch G (m x r), Q (n x r, orthonormal, B = A^T G =
    Q R), R (r x r), A Q (m x r) and a device status word (0, or k + 1 on a
    non-positive Cholesky pivot).  Rank-r approximation: (A Q) Q^T."""
    m, n = A.shape
    dev = A.device
    G = torch.empty((m, r), dtype=torch.float64, device=dev)
    Q = torch.empty((n, r), dtype=torch.float64, device=dev)
    R = torch.empty((r, r), dtype=torch.float64, device=dev)
    AQ = torch.empty((m, r), dtype=torch.float64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    check(_lib.load().genp_lowrank(m, n, _ptr(A), _ld(A), r, kind, seed, stream_id, _ptr(G), r, _ptr(Q), r, _ptr(R),
                                   r, _ptr(AQ), r, _ptr(st), _stream(stream)), "genp_lowrank")
    return G, Q, R, AQ, st


def numerical_rank(A: torch.Tensor, r_lo: int, r_hi: int, cond_max: float = 1e6, seed: int = 0, stream_id: int = 0,
                   stream=None):
    """genp_numerical_rank: (rank, B = A^T G_rank as an n x rank tensor)."""
    m, n = A.shape
    B = torch.zeros((n, max(r_hi, 1)), dtype=torch.float64, device=A.device)
    rk = ctypes.c_int64(-1)
    check(_lib.load().genp_numerical_rank(m, n, _ptr(A), _ld(A), r_lo, r_hi, float(cond_max), seed, stream_id,
                                          ctypes.byref(rk), _ptr(B), B.stride(0), _stream(stream)),
          "genp_numerical_rank")
    return int(rk.value), B[:, :int(rk.value)]
