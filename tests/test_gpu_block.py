"""Block Gaussian elimination with explicit pivot-block inverses on the GPU
(genp_block_factor; Sec. 2, Theorem 2.2's block form) against the oracle's
block_genp, through the C ABI.

* integer block factors C = L0 D U0 (identity diagonal blocks in L0 and U0,
  unimodular integer pivot blocks D_k): every step is exact in FP64, so the
  GPU's L_B, U_B and the solves agree with the oracle bit for bit;
* Gaussian-multiplied inputs: ||L_B U_B - C||_F within the normwise bound of
  block LU with explicitly inverted pivot blocks (Higham, Accuracy and
  Stability, Thm. 13.6 and the remark after it: d_n u (||C|| + ||L||||U||)
  times the pivot blocks' condition), and the solution of L_B U_B y = b
  within the first-order forward bound of the oracle's;
* the method on the n = 256 leading-singular workload to eta <= 1e-14
  (classic refinement and GMRES-IR), the adjoint within 1e-10 of the oracle
  gradient, breakdown reported at the right global step.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
U = 2.0 ** -53


@pytest.fixture(scope="module")
def g(genp_lib):
    import paper_1212_4560_gb300 as genp
    return genp


def cu(a):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV, torch.float64)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def _bidiagonal_pair(rng, k, d=None):
    """Unit lower and upper bidiagonal integer factors (off-diagonals in
    {-1, 0, 1}, U's diagonal d or random signs): their inverses have entries
    in {-1, 0, 1}, so a pivot block L U has an integer inverse with entries
    of magnitude <= k and Gauss-Jordan on it stays exact in FP64."""
    L = np.eye(k, dtype=np.int64) + np.diag(rng.integers(-1, 2, k - 1), -1)
    U = np.diag(rng.choice([-1, 1], k) if d is None else d) + np.diag(rng.integers(-1, 2, k - 1), 1)
    return L, U


def _unimodular(rng, k):
    L, U = _bidiagonal_pair(rng, k)
    return L @ U


def _integer_block_factors(n, nb, seed):
    rng = np.random.default_rng(seed)
    blocks = [(k0, min(k0 + nb, n)) for k0 in range(0, n, nb)]
    L0 = np.eye(n, dtype=np.int64)
    U0 = np.eye(n, dtype=np.int64)
    D = np.zeros((n, n), dtype=np.int64)
    for bi, (a, b) in enumerate(blocks):
        D[a:b, a:b] = _unimodular(rng, b - a)
        for bj, (c, d) in enumerate(blocks):
            if bj < bi:
                L0[a:b, c:d] = rng.integers(-1, 2, (b - a, d - c))
            elif bj > bi:
                U0[a:b, c:d] = rng.integers(-1, 2, (b - a, d - c))
    return (L0 @ D @ U0).astype(float)


@pytest.mark.parametrize("n", [64, 130, 200])
def test_block_factor_integer_exact(g, n):
    C0 = _integer_block_factors(n, 64, n)
    LUo, Pinv, k = oracle.block_genp(C0, 64)
    assert k == -1
    C = cu(C0)
    F = g.block_factor(C)
    info = g.info_fetch(F)
    assert info.breakdown_step == -1
    assert np.array_equal(host(C), LUo)
    # the solve applies the pivot blocks' inverses exactly too
    b = np.arange(n, dtype=float)[:, None] - n / 2
    y_or = oracle.block_lu_solve(LUo, Pinv, 64, b)
    G = g.make_multiplier(g.IDENTITY, n, seed=0)
    X = torch.empty((n, 1), dtype=torch.float64, device=DEV)
    g.solve(F, G, cu(b), X)
    assert np.array_equal(host(X), y_or)


@pytest.mark.parametrize("n", [64, 257, 700])
def test_block_factor_backward_error_and_solution(g, n):
    A, _, B = (t.numpy() for t in W.lead_deficient(n, 32, 16, 2, seed=n))
    M = oracle.multiplier(0, n, seed=3)
    C0 = oracle.precondition(A, M)
    C = cu(C0)
    F = g.block_factor(C)
    info = g.info_fetch(F)
    assert info.breakdown_step == -1
    LU = host(C)
    LUo, Pinv, k = oracle.block_genp(C0, 64)
    assert k == -1
    blocks = [(k0, min(k0 + 64, n)) for k0 in range(0, n, 64)]
    Lb = np.eye(n)
    Ub = np.zeros((n, n))
    for bi, (a, b) in enumerate(blocks):
        Lb[b:, a:b] = LU[b:, a:b]
        Ub[a:b, a:] = LU[a:b, a:]
    kappa_p = max(np.linalg.cond(LUo[a:b, a:b]) for a, b in blocks)
    bound = 8 * n * U * (1 + kappa_p) * (np.linalg.norm(C0) + np.linalg.norm(Lb) * np.linalg.norm(Ub))
    assert np.linalg.norm(Lb @ Ub - C0) <= bound
    # solutions of C y = b from the two factorizations, each backward stable:
    # ||y_gpu - y_or|| <= kappa(C) (eta_gpu + eta_or) (||y||) to first order, x 2
    G = g.make_multiplier(g.IDENTITY, n, seed=0)
    Y = torch.empty((n, 2), dtype=torch.float64, device=DEV)
    g.solve(F, G, cu(B), Y)
    y = host(Y)
    y_or = oracle.block_lu_solve(LUo, Pinv, 64, B)
    eta_g = oracle.backward_error(C0, y, B)
    eta_o = oracle.backward_error(C0, y_or, B)
    kc = np.linalg.cond(C0, np.inf)
    assert np.abs(y - y_or).max() <= 2 * kc * (eta_g + eta_o) * np.abs(y_or).max()
    assert eta_g <= 10 * max(eta_o, n * U)


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("n", [256, 300])
def test_block_method_leading_singular(g, n, method):
    A, X, B = (t.numpy() for t in W.lead_deficient(n, 32, 16, 1, 0))
    Ad, Bd = cu(A), cu(B)
    G = g.make_multiplier(g.GAUSSIAN, n, seed=5)
    C = torch.empty((n, n), dtype=torch.float64, device=DEV)
    g.precondition(G, Ad, C)
    F = g.block_factor(C)
    Xd = torch.empty_like(Bd)
    g.solve(F, G, Bd, Xd)
    g.refine(Ad, F, G, Bd, Xd, tol=1e-16, max_iter=8, method=method)
    info = g.info_fetch(F)
    assert info.breakdown_step == -1
    x = host(Xd)
    assert oracle.backward_error(A, x, B) <= 1e-14
    kappa = np.linalg.cond(A, np.inf)
    xd = oracle.gepp_solve(A, B)
    assert np.abs(x - xd).max() / np.abs(xd).max() <= 1e-14 * kappa
    ref = oracle.block_solve(A, B, oracle.multiplier(0, n, seed=5), 64, refine_steps=8, tol=1e-16)
    assert np.abs(x - ref["x"]).max() <= 1e-14 * kappa * np.abs(xd).max()


def test_block_breakdown_step(g):
    """C = L0 U0 with u_70,70 = 0: the leading minor of order 71 vanishes, so
    Gauss-Jordan on the second pivot block meets a zero pivot at its step 6."""
    n, k = 150, 70
    rng = np.random.default_rng(2)
    # point factors with bidiagonal 64 x 64 diagonal blocks (so every pivot
    # block L_kk U_kk has a small integer inverse and block GE stays exact)
    # and dense off-diagonal blocks
    L0 = np.tril(rng.integers(-1, 2, (n, n)), -1) + np.eye(n, dtype=np.int64)
    U0 = np.triu(rng.integers(-1, 2, (n, n)), 1)
    d = rng.choice([-1, 1], n)
    d[k] = 0
    for a in range(0, n, 64):
        b = min(a + 64, n)
        Lk, Uk = _bidiagonal_pair(rng, b - a, d[a:b])
        L0[a:b, a:b] = Lk
        U0[a:b, a:b] = Uk
    C0 = (L0 @ U0).astype(float)
    _, _, ko = oracle.block_genp(C0, 64)
    assert ko == k
    F = g.block_factor(cu(C0))
    info = g.info_fetch(F)
    assert info.breakdown_step == k
    F2 = g.block_factor(cu(np.array([[0.0, 1.0], [1.0, 0.0]])))
    assert g.info_fetch(F2).breakdown_step == 0


def test_block_adjoint_and_refactor(g):
    n, nrhs = 200, 3
    A, _, B = (t.numpy() for t in W.shifted(1, n, nrhs, seed=9))
    A, B = A[0], B[0]
    Ad, Bd = cu(A), cu(B)
    G = g.make_multiplier(g.CIRCULANT, n, seed=2)
    C = torch.empty((n, n), dtype=torch.float64, device=DEV)
    g.precondition(G, Ad, C)
    F = g.block_factor(C)
    Xd = torch.empty_like(Bd)
    g.solve(F, G, Bd, Xd)
    g.refine(Ad, F, G, Bd, Xd, tol=1e-17, max_iter=6)
    x = host(Xd)
    dA = torch.empty((n, n), dtype=torch.float64, device=DEV)
    dB = torch.empty((n, nrhs), dtype=torch.float64, device=DEV)
    g.adjoint(F, G, 2.0 * Xd, Xd, dA, dB)
    dA_ref, dB_ref = oracle.adjoint(A, x, 2.0 * x)
    assert np.linalg.norm(host(dA) - dA_ref) <= 1e-10 * np.linalg.norm(dA_ref)
    assert np.linalg.norm(host(dB) - dB_ref) <= 1e-10 * np.linalg.norm(dB_ref)
    # a second system into the same handle
    A2 = A + 0.5 * np.eye(n)
    C2 = torch.empty((n, n), dtype=torch.float64, device=DEV)
    g.precondition(G, cu(A2), C2)
    g.refactor(F, C2)
    g.solve(F, G, Bd, Xd)
    g.refine(cu(A2), F, G, Bd, Xd, tol=1e-16, max_iter=6)
    assert oracle.backward_error(A2, host(Xd), B) <= 1e-14


def test_block_factor_rejects_other_orders(g):
    import ctypes
    lib = g._lib.load()
    C = torch.zeros((8, 8), dtype=torch.float64, device=DEV)
    out = ctypes.c_void_p()
    assert lib.genp_block_factor(ctypes.c_void_p(C.data_ptr()), 8, 8, 32, None, ctypes.byref(out)) == -7
    assert lib.genp_block_factor(None, 8, 8, 64, None, ctypes.byref(out)) == -1
