"""Seeded synthetic inputs for randomized GENP.

This module is shared by the tests, the oracle side and the GPU side, and
holds none of the method's arithmetic: it only builds the systems A x = b
that the method is asked to solve.  Random numbers come from torch's
seeded generators (CPU by default; on a CUDA device for large bench inputs,
where bit-equality with a CPU copy is not needed because the oracle then
sees the device-built input copied back).  The multiplier's random numbers
are NOT drawn here: the method draws them itself from its counter-based
generator.

Workload shapes follow the paper's test problems (Sec. 7.1: a well
conditioned system whose leading blocks are singular or ill conditioned, so
that GENP without a multiplier fails) at the sizes of the benchmark suite:

* ``lead_deficient``: A ~ N(0,1) with its leading ``lead`` x ``lead`` block
  replaced by a rank-``rank`` product of Gaussian factors (so plain GENP
  meets a zero pivot at step ``rank`` in exact arithmetic), x* ~ N(0,1),
  b = A x*.  n=256/lead 32/rank 16/1 RHS and n=8192/lead 64/rank 32/16 RHS.
* ``svd_kappa``: A = J U diag(sigma) V^T with sigma log-spaced from 1 to
  1/kappa, U and V each a product of four Householder reflectors with
  N(0,1) vectors, J the row reversal (so leading blocks are ill
  conditioned).  n=16384, kappa in {1e2, 1e4, 1e6}.
* ``batched``: ``count`` systems with n uniform in [nmin, nmax], A ~ N(0,1)
  with a_11 = 0.
* ``shifted``: ``batch`` systems A = N(0,1) + 0.1 n I.
* ``table71``: the paper-shaped Table 7.1 analogue: A = [[A11, A12],
  [A21, A22]] with A11 of numerical rank n/2-1 (a rank-(n/2-1) Gaussian
  product plus 1e-12 times a Gaussian), other blocks Gaussian.
* ``lowrank``: the inputs of Tables 7.2 and 7.3 (Sec. 7.2): A = S diag(s)
  T^T with s_j = 1/j for j <= q and 1e-10 beyond (numerical rank q,
  ||A|| = 1, kappa(A) = 1e10), S and T orthogonal, each a product of four
  Householder reflectors with N(0,1) vectors (the paper says only "random
  orthogonal").
"""
from __future__ import annotations

import torch

TAG_A, TAG_X, TAG_AUX = 1, 3, 4


def _gen(seed: int, tag: int, device="cpu") -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed((int(seed) * 1_000_003 + tag * 7919) & 0x7FFF_FFFF_FFFF_FFFF)
    return g


def _randn(shape, gen, device, dtype=torch.float64):
    return torch.randn(*shape, generator=gen, device=device, dtype=dtype)


def lead_deficient(n: int, lead: int, rank: int, nrhs: int, seed: int, device="cpu"):
    """A with a rank-deficient leading block, X*, B = A X*  (float64)."""
    ga = _gen(seed, TAG_A, device)
    A = _randn((n, n), ga, device)
    if lead > 0:
        P = _randn((lead, rank), ga, device)
        Q = _randn((rank, lead), ga, device)
        A[:lead, :lead] = P @ Q
    X = _randn((n, nrhs), _gen(seed, TAG_X, device), device)
    B = A @ X
    return A, X, B


def householder_product_apply(M: torch.Tensor, V: torch.Tensor, side: str) -> torch.Tensor:
    """M <- M H_1 ... H_k (side='right') or H_1 ... H_k M (side='left') with
    H_i = I - 2 v_i v_i^T / (v_i^T v_i), v_i = V[i]."""
    if side == "right":
        for v in V:
            w = (M @ v) * (2.0 / torch.dot(v, v))
            M = M - torch.outer(w, v)
    else:
        for v in reversed(V):
            w = (v @ M) * (2.0 / torch.dot(v, v))
            M = M - torch.outer(v, w)
    return M


def svd_kappa(n: int, kappa: float, nrhs: int, seed: int, device="cpu", reflectors: int = 4):
    """A = J U diag(sigma) V^T, sigma_i = kappa^(-i/(n-1)); X*, B = A X*."""
    ga = _gen(seed, TAG_A, "cpu")
    Uv = _randn((reflectors, n), ga, "cpu").to(device)
    Vv = _randn((reflectors, n), ga, "cpu").to(device)
    i = torch.arange(n, device=device, dtype=torch.float64)
    sigma = torch.pow(torch.tensor(float(kappa), dtype=torch.float64, device=device), -i / max(n - 1, 1))
    # diag(sigma) V^T with V = H_1..H_4 => V^T = H_4..H_1; apply on the right.
    M = torch.diag(sigma)
    M = householder_product_apply(M, Vv.flip(0), "right")      # diag(s) H_4 H_3 H_2 H_1
    M = householder_product_apply(M, Uv, "left")               # H_1 H_2 H_3 H_4 (...)
    A = M.flip(0).contiguous()                                 # J: reverse the rows
    X = _randn((n, nrhs), _gen(seed, TAG_X, "cpu"), "cpu").to(device)
    B = A @ X
    return A, X, B


def batched_sizes(count: int, nmin: int, nmax: int, seed: int):
    g = _gen(seed, TAG_AUX)
    return torch.randint(nmin, nmax + 1, (count,), generator=g).tolist()


def batched(count: int, nmin: int, nmax: int, nrhs: int, seed: int, device="cpu",
            dtype=torch.float64):
    """List of (A_i, X_i, B_i) with a_11 = 0 (plain GENP breaks down at step 0)."""
    sizes = batched_sizes(count, nmin, nmax, seed)
    ga = _gen(seed, TAG_A, device)
    gx = _gen(seed, TAG_X, device)
    out = []
    for n in sizes:
        A = _randn((n, n), ga, device)
        A[0, 0] = 0.0
        X = _randn((n, nrhs), gx, device)
        out.append((A.to(dtype), X.to(dtype), (A @ X).to(dtype)))
    return out


def shifted(batch: int, n: int, nrhs: int, seed: int, device="cpu", dtype=torch.float64):
    """Batch of A = N(0,1) + 0.1 n I with X*, B = A X*  (shapes (batch, n, n))."""
    ga = _gen(seed, TAG_A, device)
    A = _randn((batch, n, n), ga, device)
    A = A + 0.1 * n * torch.eye(n, dtype=torch.float64, device=device)
    X = _randn((batch, n, nrhs), _gen(seed, TAG_X, device), device)
    B = A @ X
    return A.to(dtype), X.to(dtype), B.to(dtype)


def table71(n: int, seed: int, device="cpu"):
    """Paper-shaped analogue of the Table 7.1 inputs (construction unstated
    in the paper): well conditioned A whose n/2 x n/2 leading block has
    numerical rank n/2 - 1."""
    ga = _gen(seed, TAG_A, device)
    h = n // 2
    A = _randn((n, n), ga, device)
    P = _randn((h, h - 1), ga, device)
    Q = _randn((h - 1, h), ga, device)
    A[:h, :h] = P @ Q / (h ** 0.5) + 1e-12 * _randn((h, h), ga, device)
    X = _randn((n, 1), _gen(seed, TAG_X, device), device)
    return A, X, A @ X


def _reflectors(n: int, gen, device, count: int = 4) -> torch.Tensor:
    """Product of ``count`` Householder reflectors I - 2 v v^T / v^T v with
    N(0,1) vectors v, formed densely (n x n, orthogonal)."""
    Q = torch.eye(n, dtype=torch.float64, device=device)
    for _ in range(count):
        v = _randn((n, 1), gen, device)
        Q = Q - (2.0 / float((v * v).sum())) * (Q @ v) @ v.T
    return Q


def lowrank(n: int, q: int, seed: int, device="cpu"):
    """Tables 7.2 / 7.3 inputs: A = S diag(s) T^T, s_j = 1/j (j <= q), 1e-10
    (j > q).  Returns A, S, T, s."""
    gs = _gen(seed, TAG_A, device)
    S = _reflectors(n, gs, device)
    T = _reflectors(n, gs, device)
    s = torch.full((n,), 1e-10, dtype=torch.float64, device=device)
    s[:q] = 1.0 / torch.arange(1, q + 1, dtype=torch.float64, device=device)
    A = (S * s) @ T.T
    return A, S, T, s
