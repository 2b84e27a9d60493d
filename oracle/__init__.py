"""CPU FP64 oracle for randomized GENP (Pan & Qian, arXiv:1212.4560).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  It shares no code with the CUDA library and never imports it;
the CUDA library never calls it.

The arithmetic lives in ``genp_oracle.c`` (plain loops in IEEE double, no
fused multiply-add).  This module loads it with ctypes, adds the pipeline of
the method (Sec. 1.1; Cor. 4.1, the ``MH`` form of Thm. 4.1 with M = A,
H = G), iterative refinement (Sec. 7.1: one refinement step in Table 7.1),
the adjoint, exact Leibniz determinants and error measures.

Parity pins live in ``tests/test_oracle_*.py``.  Parity unpinned: agreement
with the statistics of Table 7.1 (the paper does not give its matrix
construction, and its +-1 circulant is not the multiplier used here).
"""
from __future__ import annotations

import ctypes
import math
import itertools
import os
from fractions import Fraction

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64

KIND_GAUSSIAN, KIND_CIRCULANT, KIND_SPARSE, KIND_CIRCULANT_PM1, KIND_IDENTITY = 0, 1, 2, 3, 4
KIND_TOEPLITZ, KIND_HOUSEHOLDER_PM1 = 5, 6


def lib():
    """Loads (building first if needed) the oracle's shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.or_philox4x64_10.argtypes = [ctypes.POINTER(_u64), ctypes.POINTER(_u64), ctypes.POINTER(_u64)]
        L.or_u53.argtypes = [_u64]
        L.or_u53.restype = ctypes.c_double
        L.or_log.argtypes = [ctypes.c_double]
        L.or_log.restype = ctypes.c_double
        L.or_gauss.argtypes = [_u64, _u64, _u64, _u64]
        L.or_gauss.restype = ctypes.c_double
        L.or_log_f32.argtypes = [ctypes.c_float]
        L.or_log_f32.restype = ctypes.c_float
        L.or_gauss_f32.argtypes = [_u64, _u64, _u64, _u64]
        L.or_gauss_f32.restype = ctypes.c_float
        L.or_mult_dense_f32.argtypes = [_i64, _u64, _u64, ctypes.c_float, _dp, _i64]
        L.or_mult_circulant_f32.argtypes = [_i64, _u64, _u64, ctypes.c_float, _dp]
        L.or_mult_dense.argtypes = [_i64, _u64, _u64, ctypes.c_double, _dp, _i64]
        L.or_mult_circulant.argtypes = [_i64, _u64, _u64, ctypes.c_double, _dp]
        L.or_mult_circulant_pm1.argtypes = [_i64, _u64, _u64, _dp]
        L.or_mult_circulant_pm1.restype = ctypes.c_int
        L.or_circulant_pm1_singular.argtypes = [_i64, _dp]
        L.or_circulant_pm1_singular.restype = ctypes.c_int
        L.or_mult_sparse.argtypes = [_i64, ctypes.c_int, _u64, _u64, ctypes.c_void_p, ctypes.c_void_p]
        L.or_circulant_to_dense.argtypes = [_i64, _dp, _dp, _i64]
        L.or_mult_toeplitz.argtypes = [_i64, _u64, _u64, ctypes.c_double, _dp]
        L.or_mult_toeplitz_f32.argtypes = [_i64, _u64, _u64, ctypes.c_float, _dp]
        L.or_toeplitz_to_dense.argtypes = [_i64, _dp, _dp, _i64]
        L.or_mult_householder_pm1.argtypes = [_i64, _u64, _u64, _dp]
        L.or_mult_sketch.argtypes = [_i64, _i64, ctypes.c_int, _u64, _u64, ctypes.c_double, _dp, _i64]
        L.or_householder_to_dense.argtypes = [_i64, _dp, _dp, _i64]
        L.or_sparse_to_dense.argtypes = [_i64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, _dp, _i64]
        L.or_matmul.argtypes = [_i64, _i64, _i64, _dp, _i64, _dp, _i64, _dp, _i64]
        L.or_genp.argtypes = [_i64, _dp, _i64]
        L.or_genp.restype = _i64
        L.or_gepp.argtypes = [_i64, _dp, _i64, ctypes.c_void_p]
        L.or_gepp.restype = _i64
        for f in ("or_solve_lower_unit", "or_solve_upper", "or_solve_upper_T", "or_solve_lower_unit_T"):
            getattr(L, f).argtypes = [_i64, _i64, _dp, _i64, _dp, _i64]
        L.or_apply_piv.argtypes = [_i64, _i64, ctypes.c_void_p, _dp, _i64]
        L.or_apply_piv_T.argtypes = [_i64, _i64, ctypes.c_void_p, _dp, _i64]
        L.or_residual.argtypes = [_i64, _i64, _dp, _i64, _dp, _i64, _dp, _i64, _dp, _i64]
        L.or_backward_error.argtypes = [_i64, _i64, _dp, _i64, _dp, _i64, _dp, _i64]
        L.or_backward_error.restype = ctypes.c_double
        L.or_circ_matmul.argtypes = [_i64, _i64, _dp, _i64, _dp, _dp, _i64]
        L.or_sparse_matmul.argtypes = [_i64, _i64, ctypes.c_int, _dp, _i64, ctypes.c_void_p,
                                       ctypes.c_void_p, _dp, _i64]
        L.or_circ_apply.argtypes = [_i64, _i64, ctypes.c_int, _dp, _dp, _i64, _dp, _i64]
        L.or_gauss_jordan_inverse.argtypes = [_i64, _dp, _i64, _dp, _i64]
        L.or_gauss_jordan_inverse.restype = _i64
        L.or_block_genp.argtypes = [_i64, _dp, _i64, _i64, _dp]
        L.or_block_genp.restype = _i64
        L.or_block_lu_solve.argtypes = [_i64, _i64, _dp, _i64, _i64, _dp, _dp, _i64]
        L.or_sparse_apply.argtypes = [_i64, _i64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.c_void_p, _dp, _i64, _dp, _i64]
        _lib = L
    return _lib


def _c(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


# --------------------------------------------------------------------------
# Random numbers and multipliers
# --------------------------------------------------------------------------

def philox4x64_10(ctr, key) -> np.ndarray:
    """One Philox4x64-10 block (Salmon et al., SC'11) for counter and key."""
    c = (_u64 * 4)(*[int(x) & (2**64 - 1) for x in ctr])
    k = (_u64 * 2)(*[int(x) & (2**64 - 1) for x in key])
    o = (_u64 * 4)()
    lib().or_philox4x64_10(c, k, o)
    return np.array(list(o), dtype=np.uint64)


def log(s: float) -> float:
    """The oracle's own natural log (atanh series), positive normal input."""
    return lib().or_log(float(s))


def gauss(seed: int, stream: int, tag: int, idx: int) -> float:
    return lib().or_gauss(seed, stream, tag, idx)


def log_f32(s: float) -> float:
    return lib().or_log_f32(float(s))


def gauss_f32(seed: int, stream: int, tag: int, idx: int) -> float:
    return lib().or_gauss_f32(seed, stream, tag, idx)


def multiplier(kind: int, n: int, seed: int, stream: int = 0, scale: float | None = None,
               nnz: int = 4, grid: str = "fp64"):
    """The random multiplier G (Definition 3.2 / Sec. 2.3 / sparse reading).
    Kinds: 0 Gaussian, 1 Gaussian circulant, 2 sparse +-1, 3 circulant with a
    +-1 first column (the paper's test multiplier, Sec. 7.1; redrawn until its
    power-of-two-order DFT bins are nonzero), 4 the identity (plain GENP),
    5 Gaussian Toeplitz (Definition 3.2; ``t`` holds t_{-(n-1)} .. t_{n-1}),
    6 Householder reflector I - 2 u u^T / n with a +-1 vector ``u`` (the
    Householder multipliers of Sec. 7.1, read as an orthogonal reflector).

    grid "fp64": entries drawn in double precision; "fp32": drawn by the same
    polar method in single precision (scale rounded to float first).
    Returns a dict with the structure (``G`` dense n x n always, plus ``g``
    for a circulant, ``rows``/``signs`` for the sparse multiplier)."""
    L = lib()
    if kind == KIND_GAUSSIAN:
        s = (1.0 / np.sqrt(float(n))) if scale is None else float(scale)
        G = np.empty((n, n))
        if grid == "fp32":
            L.or_mult_dense_f32(n, seed, stream, float(np.float32(s)), _p(G), n)
        else:
            L.or_mult_dense(n, seed, stream, s, _p(G), n)
        return {"kind": kind, "n": n, "G": G}
    if kind == KIND_CIRCULANT:
        s = 1.0 if scale is None else float(scale)
        g = np.empty(n)
        if grid == "fp32":
            L.or_mult_circulant_f32(n, seed, stream, float(np.float32(s)), _p(g))
        else:
            L.or_mult_circulant(n, seed, stream, s, _p(g))
        out = {"kind": kind, "n": n, "g": g}
        if n <= 4096:
            G = np.empty((n, n))
            L.or_circulant_to_dense(n, _p(g), _p(G), n)
            out["G"] = G
        return out
    if kind == KIND_CIRCULANT_PM1:
        g = np.empty(n)
        attempt = L.or_mult_circulant_pm1(n, seed, stream, _p(g))
        out = {"kind": kind, "n": n, "g": g, "attempt": int(attempt)}
        if n <= 4096:
            G = np.empty((n, n))
            L.or_circulant_to_dense(n, _p(g), _p(G), n)
            out["G"] = G
        return out
    if kind == KIND_IDENTITY:
        return {"kind": kind, "n": n, "G": np.eye(n)}
    if kind == KIND_TOEPLITZ:
        s = 1.0 if scale is None else float(scale)
        t = np.empty(2 * n - 1)
        if grid == "fp32":
            L.or_mult_toeplitz_f32(n, seed, stream, float(np.float32(s)), _p(t))
        else:
            L.or_mult_toeplitz(n, seed, stream, s, _p(t))
        out = {"kind": kind, "n": n, "t": t}
        if n <= 8192:      # products below use the dense matrix (the plain definition)
            G = np.empty((n, n))
            L.or_toeplitz_to_dense(n, _p(t), _p(G), n)
            out["G"] = G
        return out
    if kind == KIND_HOUSEHOLDER_PM1:
        u = np.empty(n)
        L.or_mult_householder_pm1(n, seed, stream, _p(u))
        out = {"kind": kind, "n": n, "u": u}
        if n <= 8192:
            G = np.empty((n, n))
            L.or_householder_to_dense(n, _p(u), _p(G), n)
            out["G"] = G
        return out
    if kind == KIND_SPARSE:
        rows = np.empty((nnz, n), dtype=np.int32)
        signs = np.empty((nnz, n), dtype=np.int8)
        L.or_mult_sparse(n, nnz, seed, stream, rows.ctypes.data, signs.ctypes.data)
        out = {"kind": kind, "n": n, "rows": rows, "signs": signs, "nnz": nnz}
        if n <= 4096:
            G = np.empty((n, n))
            L.or_sparse_to_dense(n, nnz, rows.ctypes.data, signs.ctypes.data, _p(G), n)
            out["G"] = G
        return out
    raise ValueError(kind)


def circulant_pm1_singular(g) -> bool:
    """The exact integer singularity test of the +-1 circulant draw."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    return bool(lib().or_circulant_pm1_singular(len(g), _p(g)))


# --------------------------------------------------------------------------
# The method's steps
# --------------------------------------------------------------------------

def matmul(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    A, B = _c(A), _c(B)
    m, k = A.shape
    n = B.shape[1]
    C = np.empty((m, n))
    lib().or_matmul(m, k, n, _p(A), k, _p(B), n, _p(C), n)
    return C


def precondition(A: np.ndarray, M: dict, rows=None) -> np.ndarray:
    """C = A G (Thm. 4.1, the MH product), by the definition of each kind.

    ``rows`` restricts the product to a subset of rows of A (for sampled
    checks at sizes where the full product is too slow)."""
    A = _c(A if rows is None else A[rows])
    m, n = A.shape
    C = np.empty((m, M["n"]))
    L = lib()
    if M["kind"] in (KIND_GAUSSIAN, KIND_TOEPLITZ, KIND_HOUSEHOLDER_PM1):
        return matmul(A, M["G"])
    if M["kind"] == KIND_IDENTITY:
        return A.copy()
    if M["kind"] in (KIND_CIRCULANT, KIND_CIRCULANT_PM1):
        L.or_circ_matmul(m, n, _p(A), n, _p(_c(M["g"])), _p(C), n)
        return C
    L.or_sparse_matmul(m, n, M["nnz"], _p(A), n, M["rows"].ctypes.data, M["signs"].ctypes.data,
                       _p(C), n)
    return C


def precondition_left(A: np.ndarray, M: dict) -> np.ndarray:
    """C = G A, the GM half of Thm. 4.1 / Cor. 4.1 (the multiplier on the
    left), by the definition: the product with the dense G."""
    if M["kind"] == KIND_IDENTITY:
        return _c(A).copy()
    return matmul(M["G"], _c(A))


def apply_multiplier(M: dict, Y: np.ndarray, trans: bool = False) -> np.ndarray:
    """X = G Y (or G^T Y), Y of shape (n, nrhs), by the definition of G."""
    Y = _c(Y)
    n, nrhs = Y.shape
    X = np.empty_like(Y)
    L = lib()
    if M["kind"] in (KIND_GAUSSIAN, KIND_TOEPLITZ, KIND_HOUSEHOLDER_PM1):
        return matmul(M["G"].T.copy() if trans else M["G"], Y)
    if M["kind"] == KIND_IDENTITY:
        return Y.copy()
    if M["kind"] in (KIND_CIRCULANT, KIND_CIRCULANT_PM1):
        L.or_circ_apply(n, nrhs, int(trans), _p(_c(M["g"])), _p(Y), nrhs, _p(X), nrhs)
        return X
    L.or_sparse_apply(n, nrhs, int(trans), M["nnz"], M["rows"].ctypes.data, M["signs"].ctypes.data,
                      _p(Y), nrhs, _p(X), nrhs)
    return X


def genp(C: np.ndarray):
    """Unblocked GENP (Sec. 1.1), in place on a copy.  Returns (LU, step)
    with step = -1 on success, else the first zero / non-finite pivot."""
    LU = _c(C).copy()
    n = LU.shape[0]
    k = lib().or_genp(n, _p(LU), n)
    return LU, int(k)


def gepp(A: np.ndarray):
    """GEPP with first-max tie-break.  Returns (LU, piv, step)."""
    LU = _c(A).copy()
    n = LU.shape[0]
    piv = np.zeros(n, dtype=np.int64)
    k = lib().or_gepp(n, _p(LU), n, piv.ctypes.data)
    return LU, piv, int(k)


def split_lu(LU: np.ndarray):
    L = np.tril(LU, -1) + np.eye(LU.shape[0])
    U = np.triu(LU)
    return L, U


def lu_solve(LU: np.ndarray, B: np.ndarray) -> np.ndarray:
    """y = U^{-1} L^{-1} B by forward then back substitution."""
    Y = _c(B).copy()
    if Y.ndim == 1:
        Y = Y[:, None]
    n, nrhs = Y.shape
    L = lib()
    L.or_solve_lower_unit(n, nrhs, _p(LU), n, _p(Y), nrhs)
    L.or_solve_upper(n, nrhs, _p(LU), n, _p(Y), nrhs)
    return Y


def lu_solve_T(LU: np.ndarray, B: np.ndarray) -> np.ndarray:
    """y = L^{-T} U^{-T} B."""
    Y = _c(B).copy()
    n, nrhs = Y.shape
    L = lib()
    L.or_solve_upper_T(n, nrhs, _p(LU), n, _p(Y), nrhs)
    L.or_solve_lower_unit_T(n, nrhs, _p(LU), n, _p(Y), nrhs)
    return Y


def gepp_solve(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Definition-level solution x = A^{-1} B by GEPP (no multiplier)."""
    LU, piv, k = gepp(A)
    if k >= 0:
        raise np.linalg.LinAlgError(f"singular at step {k}")
    Y = _c(B).copy()
    if Y.ndim == 1:
        Y = Y[:, None]
    n, nrhs = Y.shape
    lib().or_apply_piv(n, nrhs, piv.ctypes.data, _p(Y), nrhs)
    return lu_solve(LU, Y)


def gepp_solve_T(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """x = A^{-T} B by GEPP on A^T (independent of any multiplier)."""
    return gepp_solve(_c(A).T.copy(), B)


def residual(A, X, B) -> np.ndarray:
    A, X, B = _c(A), _c(X), _c(B)
    n, nrhs = X.shape
    R = np.empty_like(X)
    lib().or_residual(n, nrhs, _p(A), n, _p(X), nrhs, _p(B), nrhs, _p(R), nrhs)
    return R


def backward_error(A, X, B) -> float:
    """max over columns of ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)."""
    A, X, B = _c(A), _c(X), _c(B)
    if X.ndim == 1:
        X, B = X[:, None], B[:, None]
    n, nrhs = X.shape
    return lib().or_backward_error(n, nrhs, _p(A), n, _p(X), nrhs, _p(B), nrhs)


def rel_residual_2(A, X, B) -> float:
    """Table 7.1's measure ||A y - b|| / ||b|| in the 2-norm (Sec. 2.4)."""
    R = residual(A, _c(X).reshape(len(X), -1), _c(B).reshape(len(B), -1))
    return float(np.linalg.norm(R) / np.linalg.norm(B))


def solve(A: np.ndarray, B: np.ndarray, M: dict, refine_steps: int = 0, tol: float = 0.0, side: str = "right"):
    """The whole method: C = A G, GENP(C), y = U^-1 L^-1 b, x = G y, then up
    to ``refine_steps`` refinement steps r = b - A x, C d = r, x += G d,
    stopping early when the backward error reaches ``tol`` or stops halving.
    side "left": C = G A, GENP(C), x = U^-1 L^-1 (G b), and the refinement
    steps d = U^-1 L^-1 (G r), x += d.

    Returns dict(x, LU, step, eta) with eta the backward errors after the
    solve and after each refinement step."""
    B2 = _c(B).reshape(B.shape[0], -1)
    left = side == "left"
    C = precondition_left(A, M) if left else precondition(A, M)
    LU, step = genp(C)
    out = {"LU": LU, "step": step, "C": C}
    if step >= 0:
        out.update(x=None, eta=[np.inf])
        return out
    if left:
        X = lu_solve(LU, apply_multiplier(M, B2))
    else:
        X = apply_multiplier(M, lu_solve(LU, B2))
    eta = [backward_error(A, X, B2)]
    for _ in range(refine_steps):
        if eta[-1] <= tol:
            break
        R = residual(A, X, B2)
        D = lu_solve(LU, apply_multiplier(M, R)) if left else apply_multiplier(M, lu_solve(LU, R))
        X = X + D
        eta.append(backward_error(A, X, B2))
        if eta[-1] > eta[-2] / 2:
            break
    out.update(x=X, eta=eta)
    return out


def gauss_jordan_inverse(P: np.ndarray):
    """P^{-1} by Gauss-Jordan elimination without pivoting.  Returns (X, step)
    with step = -1, or the first zero / non-finite pivot."""
    P = _c(P)
    kb = P.shape[0]
    X = np.zeros((kb, kb))
    t = lib().or_gauss_jordan_inverse(kb, _p(P), kb, _p(X), kb)
    return X, int(t)


def block_genp(C: np.ndarray, nb: int):
    """Block Gaussian elimination with explicit inverses of the pivot blocks
    (Sec. 2, the block form of Theorem 2.2), in place on a copy.  Returns
    (LU, Pinv, step): LU holds L_B below the block diagonal and U_B on and
    above it (pivot blocks on the diagonal), Pinv[k] the nb x nb slot of
    P_k^{-1} (top-left kb x kb for a ragged last block), step -1 or the first
    zero / non-finite pivot."""
    LU = _c(C).copy()
    n = LU.shape[0]
    nblk = (n + nb - 1) // nb
    Pinv = np.zeros((nblk, nb, nb))
    k = lib().or_block_genp(n, _p(LU), n, nb, _p(Pinv))
    return LU, Pinv, int(k)


def block_lu_solve(LU: np.ndarray, Pinv: np.ndarray, nb: int, B: np.ndarray) -> np.ndarray:
    """y = U_B^{-1} L_B^{-1} B: block forward substitution, then block back
    substitution through the pivot blocks' inverses."""
    Y = _c(B).copy()
    if Y.ndim == 1:
        Y = Y[:, None]
    n, nrhs = Y.shape
    lib().or_block_lu_solve(n, nrhs, _p(LU), n, nb, _p(_c(Pinv)), _p(Y), nrhs)
    return Y


def block_solve(A: np.ndarray, B: np.ndarray, M: dict, nb: int, refine_steps: int = 0, tol: float = 0.0):
    """The method with block GE in place of GENP: C = A G, block GE of C,
    y = U_B^-1 L_B^-1 b, x = G y, then FP64 refinement r = b - A x,
    C d = r, x += G d (stopping as in ``solve``).  Returns dict(x, LU, Pinv,
    step, eta)."""
    B2 = _c(B).reshape(B.shape[0], -1)
    C = precondition(A, M)
    LU, Pinv, step = block_genp(C, nb)
    out = {"LU": LU, "Pinv": Pinv, "step": step, "C": C}
    if step >= 0:
        out.update(x=None, eta=[np.inf])
        return out
    X = apply_multiplier(M, block_lu_solve(LU, Pinv, nb, B2))
    eta = [backward_error(A, X, B2)]
    for _ in range(refine_steps):
        if eta[-1] <= tol:
            break
        R = residual(A, X, B2)
        X = X + apply_multiplier(M, block_lu_solve(LU, Pinv, nb, R))
        eta.append(backward_error(A, X, B2))
        if eta[-1] > eta[-2] / 2:
            break
    out.update(x=X, eta=eta)
    return out


def adjoint(A: np.ndarray, X: np.ndarray, gX: np.ndarray):
    """Gradient of a loss l(X) with X = A^{-1} B given gX = dl/dX:
    lambda = A^{-T} gX (by GEPP on A^T, independent of the multiplier),
    dA = -lambda X^T, dB = lambda."""
    lam = gepp_solve_T(A, gX)
    dA = -matmul(lam, _c(X).T.copy())
    return dA, lam


# --------------------------------------------------------------------------
# Randomized low-rank approximation (Sec. 5, Proto-Alg. 5.1; Sec. 7.2)
# --------------------------------------------------------------------------

def sketch_multiplier(m: int, r: int, seed: int, stream: int = 0, toeplitz: bool = False,
                      scale: float = 1.0) -> np.ndarray:
    """The m x r multiplier of Stage 1: Gaussian G_{0,scale}^{m x r}, or the
    Gaussian Toeplitz matrix of Table 7.3."""
    G = np.empty((m, r))
    lib().or_mult_sketch(m, r, int(toeplitz), seed, stream, float(scale), _p(G), r)
    return G


def lowrank_approx(A: np.ndarray, G: np.ndarray):
    """Proto-Alg. 5.1 with an orthonormal T as in the tests of Sec. 7.2:
    Stage 1 T' = A^T G; the orthonormal factor Q of T' = Q R with a
    positive diagonal of R (Fact 2.2: then Q is unique), by a library QR with
    the column signs fixed; Stage 3 A_hat = A T (T^T T)^{-1} T^T = (A Q) Q^T.
    Returns dict(B = A^T G, Q, AQ)."""
    A = _c(A)
    B = matmul(A.T.copy(), _c(G))
    Q, R = np.linalg.qr(B, mode="reduced")
    sgn = np.where(np.diag(R) < 0, -1.0, 1.0)
    Q = Q * sgn[None, :]
    return {"B": B, "Q": Q, "AQ": matmul(A, Q)}


def lowrank_residuals(A: np.ndarray, B: np.ndarray, Q: np.ndarray, AQ: np.ndarray, T_lead: np.ndarray):
    """The residual norms of Tables 7.2 / 7.3 (2-norms, Sec. 2.4):
    rn1 = ||B Y - T_lead|| with Y the least-squares solution (B's columns
    approximate the leading right singular space of A, spanned by T_lead);
    rn2 = ||A - A Q Q^T||."""
    Y = np.linalg.lstsq(B, T_lead, rcond=None)[0]
    rn1 = float(np.linalg.norm(B @ Y - T_lead, 2))
    rn2 = float(np.linalg.norm(_c(A) - AQ @ Q.T, 2))
    return rn1, rn2


def numerical_rank(A: np.ndarray, r_lo: int, r_hi: int, cond_max: float, G: np.ndarray):
    """App. B, Proto-Alg. B.1 (numerical rank without pivoting or
    orthogonalization), as read here: with the m x r_hi Gaussian G drawn once
    and G_r its first r columns, the sketch B' = A^T G_r is full rank and
    well conditioned exactly when r does not exceed the numerical rank
    (Thm. 5.1), so the rank is the largest r in [r_lo, r_hi] whose sketch
    passes COND; binary search r = ceil((r_lo + r_hi) / 2) (Remark B.4):
    pass -> r_lo = r, fail -> r_hi = r - 1.  COND: kappa_2(B') <= cond_max
    (here by the library SVD).  Returns (rank, B = A^T G_rank, trace of
    (r, kappa, passed) per test)."""
    A, G = _c(A), _c(G)
    lo, hi = int(r_lo), int(r_hi)
    trace = []
    while lo < hi:
        r = (lo + hi + 1) // 2
        Bp = matmul(A.T.copy(), G[:, :r].copy())
        kappa = float(np.linalg.cond(Bp))
        ok = bool(np.isfinite(kappa) and kappa <= cond_max)
        trace.append((r, kappa, ok))
        if ok:
            lo = r
        else:
            hi = r - 1
    B = matmul(A.T.copy(), G[:, :lo].copy()) if lo > 0 else np.zeros((A.shape[1], 0))
    return lo, B, trace


# --------------------------------------------------------------------------
# FP8 (e4m3) operands with a power-of-two scale per 128 x 128 tile (the
# mixed-precision pattern: Schur update and A G on 8-bit operands, accuracy
# won back by FP64 refinement, Sec. 7.1)
# --------------------------------------------------------------------------

E4M3_MAX = 448.0          # 1.75 * 2^8, the largest finite e4m3 value
FP8_TILE = 128


def e4m3_decode(codes) -> np.ndarray:
    """Value of each e4m3 code (1 sign bit, 4 exponent bits with bias 7, 3
    mantissa bits; exponent field 0 is subnormal, m/8 * 2^-6; code S.1111.111
    is NaN; there are no infinities)."""
    c = np.asarray(codes, dtype=np.int64)
    sgn = np.where(c & 0x80, -1.0, 1.0)
    E = (c >> 3) & 0xF
    m = (c & 7).astype(np.float64)
    v = np.where(E == 0, m / 8.0 * 2.0 ** -6, (1.0 + m / 8.0) * np.exp2(E.astype(np.float64) - 7.0))
    v = np.where((E == 15) & ((c & 7) == 7), np.nan, v)
    return sgn * v


def e4m3_round(x) -> np.ndarray:
    """Nearest e4m3 value of each (finite) x, ties to the even mantissa,
    magnitudes above 448 saturated to 448.  Below 2^-6 the spacing is the
    subnormal quantum 2^-9; in [2^p, 2^{p+1}) it is 2^{p-3}."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    _, p = np.frexp(a)                       # a = f 2^p, f in [0.5, 1): binade 2^{p-1}
    qexp = np.maximum(p - 1, -6) - 3
    q = np.ldexp(np.rint(np.ldexp(a, -qexp)), qexp)    # rint: ties to even
    q = np.minimum(q, E4M3_MAX)
    return np.copysign(q, x)


def e4m3_encode(v) -> np.ndarray:
    """Code of each value already on the e4m3 grid (inverse of e4m3_decode)."""
    v = np.asarray(v, dtype=np.float64)
    a = np.abs(v)
    sign = np.where(np.signbit(v), 0x80, 0)
    _, p = np.frexp(a)
    normal = a >= 2.0 ** -6
    E = np.where(normal, p - 1 + 7, 0)
    m = np.where(normal, np.ldexp(a, -(p - 1)) * 8.0 - 8.0, np.ldexp(a, 9))
    return (sign | (E << 3) | m.astype(np.int64)).astype(np.uint8)


def tile_exponent(amax: float) -> int:
    """The least integer e with amax <= 448 2^e (0 for amax = 0), clamped to
    [-126, 126] so that 2^e is a normal FP32 number.  With amax = f 2^p,
    f in [0.5, 1): 448 2^e = 0.875 2^{e+9}, so e = p - 9 when f <= 0.875,
    else p - 8."""
    if not (amax > 0.0) or not np.isfinite(amax):
        return 0
    f, p = np.frexp(float(amax))
    e = int(p) - 9 if f <= 0.875 else int(p) - 8
    return max(-126, min(126, e))


def quantize_e4m3(X: np.ndarray):
    """Codes and scales of X (m x K) with one power-of-two scale per
    128 x 128 tile (tile (ti, kt): rows 128 ti .., columns 128 kt ..):
    codes[i, k] = e4m3(X[i, k] / 2^e_tile), scales[ti, kt] = 2^e_tile."""
    X = np.asarray(X, dtype=np.float64)
    m, K = X.shape
    T = FP8_TILE
    ntm, nkt = -(-m // T), -(-K // T)
    codes = np.zeros((m, K), dtype=np.uint8)
    scales = np.ones((ntm, nkt))
    for ti in range(ntm):
        for kt in range(nkt):
            blk = X[ti * T:(ti + 1) * T, kt * T:(kt + 1) * T]
            e = tile_exponent(float(np.max(np.abs(blk))) if blk.size else 0.0)
            scales[ti, kt] = 2.0 ** e
            codes[ti * T:(ti + 1) * T, kt * T:(kt + 1) * T] = e4m3_encode(e4m3_round(np.ldexp(blk, -e)))
    return codes, scales


def dequantize_e4m3(codes: np.ndarray, scales: np.ndarray) -> np.ndarray:
    """The values the codes and tile scales stand for."""
    T = FP8_TILE
    S = np.repeat(np.repeat(scales, T, axis=0), T, axis=1)[: codes.shape[0], : codes.shape[1]]
    return e4m3_decode(codes) * S


def gemm_e4m3(Aq, sA, Bq, sB, alpha: float = 1.0, beta: float = 0.0, C=None) -> np.ndarray:
    """D = alpha sum_kt sA[tm, kt] sB[tn, kt] (A_kt B_kt^T) + beta C, for
    A (m x K) and B^T (n x K) as codes with tile scales.  Each k-tile's
    products of e4m3 values and their sums are exact in FP64 (at most 43
    significant bits); the k-tiles are summed in FP64."""
    T = FP8_TILE
    A = e4m3_decode(Aq)
    B = e4m3_decode(Bq)
    m, K = A.shape
    n = B.shape[0]
    D = np.zeros((m, n))
    for kt in range(-(-K // T)):
        P = matmul(A[:, kt * T:(kt + 1) * T].copy(), B[:, kt * T:(kt + 1) * T].T.copy())
        rs = np.repeat(sA[:, kt], T)[:m]
        cs = np.repeat(sB[:, kt], T)[:n]
        D += P * rs[:, None] * cs[None, :]
    D *= alpha
    if beta != 0.0:
        D += beta * np.asarray(C, dtype=np.float64)
    return D


def genp_fp8(C: np.ndarray, nb: int = 128):
    """Blocked GENP (the block form of Thm. 2.2) with the Schur complement
    update on e4m3 operands, everything else in FP64: for each nb-wide step,
    the diagonal block by unblocked GENP, the block row U12 = L11^{-1} C12
    and the block column L21 = C21 U11^{-1} by substitution, then
    C22 -= deq(q(L21)) deq(q(U12^T))^T, with q the tile-scaled e4m3
    quantization (tiles counted from each operand's own origin) and the
    product of the dequantized operands exact per k-tile (gemm_e4m3).
    Returns (LU, step) as genp does."""
    LU = _c(C).copy()
    n = LU.shape[0]
    L = lib()
    step = -1
    for k0 in range(0, n, nb):
        kb = min(nb, n - k0)
        D, s = genp(LU[k0:k0 + kb, k0:k0 + kb])
        LU[k0:k0 + kb, k0:k0 + kb] = D
        if s >= 0 and step < 0:
            step = k0 + s
        rem = n - k0 - kb
        if rem == 0:
            break
        U12 = _c(LU[k0:k0 + kb, k0 + kb:]).copy()          # L11^{-1} C12
        L.or_solve_lower_unit(kb, rem, _p(D), kb, _p(U12), rem)
        L21t = _c(LU[k0 + kb:, k0:k0 + kb].T).copy()       # (C21 U11^{-1})^T = U11^{-T} C21^T
        L.or_solve_upper_T(kb, rem, _p(D), kb, _p(L21t), rem)
        LU[k0:k0 + kb, k0 + kb:] = U12
        LU[k0 + kb:, k0:k0 + kb] = L21t.T
        qa, sa = quantize_e4m3(L21t.T)
        qb, sb = quantize_e4m3(U12.T)
        LU[k0 + kb:, k0 + kb:] -= gemm_e4m3(qa, sa, qb, sb)
    return LU, step


FP8_GRID_SD = 12.5        # bounds every polar-method draw (|z| <= sqrt(2 ln 2^104) < 12.1)


def fp8_grid(G: np.ndarray, scale: float) -> np.ndarray:
    """A Gaussian multiplier of entry scale ``scale`` rounded to the FP8 grid:
    e4m3 values times 2^e, e = tile_exponent(12.5 scale), one exponent for the
    whole matrix (Thm. 4.1 admits the perturbation; the rounded G is the
    multiplier everywhere, so G A and x = G y use the same matrix).  G is the
    FP32-grid draw (``multiplier(..., grid="fp32")``): the FP8 grid rounds
    that draw."""
    e = tile_exponent(FP8_GRID_SD * float(scale))
    return np.ldexp(e4m3_round(np.ldexp(np.asarray(G, dtype=np.float64), -e)), e)


# --------------------------------------------------------------------------
# Exact references used by the pins
# --------------------------------------------------------------------------

def sliced_grid_exponent(scale: float) -> int:
    """E, the least integer with 12.5 scale <= 2^E (12.5 standard deviations
    bound every polar draw)."""
    amax = 12.5 * float(scale)
    if not amax > 0.0:
        return 0
    f, p = math.frexp(amax)
    return p - 1 if f == 0.5 else p


def sliced_grid(G: np.ndarray, scale: float, digits: int = 2) -> np.ndarray:
    """The multiplier rounded to the fixed-point grid of the sliced product
    with ``digits`` balanced 7-bit digits: the nearest integer multiple of
    2^(E - 7 digits + 1), ties to even (Thm. 4.1's perturbed Gaussian
    G = G' + U with |U| <= 2^(E - 7 digits)): 2^(E - 13) for two digits,
    2^(E - 6) for one.  The library rounds its single precision draw
    (``multiplier(..., grid="fp32")``)."""
    if digits not in (1, 2):
        raise ValueError("digits: 1 or 2")
    E = sliced_grid_exponent(scale)
    q = 7 * digits - 1
    return np.ldexp(np.rint(np.ldexp(_c(G), q - E)), E - q)


def det_leibniz(M) -> Fraction:
    """det(M) = sum over permutations of sign(p) prod_i m[i, p(i)], exact in
    rationals (every double is a rational).  n <= 7."""
    n = len(M)
    F = [[Fraction(float(M[i][j])) for j in range(n)] for i in range(n)]
    total = Fraction(0)
    for perm in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if perm[i] > perm[j])
        term = Fraction(-1 if inv % 2 else 1)
        for i in range(n):
            term *= F[i][perm[i]]
            if term == 0:
                break
        total += term
    return total
