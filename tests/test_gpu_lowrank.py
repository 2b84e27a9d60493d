"""Randomized low-rank approximation (Sec. 5, Proto-Alg. 5.1) on the GPU
vs the CPU oracle, through the C ABI.

Tolerances (u = 2^-53):
* the sketch G: bit-exact (same Philox counters, same polar method);
* B = A^T G (FP64 GEMM): |dB| <= 2 gamma_m |A|^T |G|;
* Q: unique (B = Q R, R with a positive diagonal), so compared entry by
  entry with the oracle's: ||dQ||_2 <= 1e3 n r u kappa(B) (both QR
  factorizations are backward stable; Q's perturbation is bounded by
  kappa(B) times the backward error, Higham Thm. 19.4 / 19.10);
* orthogonality ||Q^T Q - I|| <= 100 n r u (CholeskyQR3 reaches Householder
  level for kappa(B) below 1/u);
* residual norms of Tables 7.2 / 7.3 within 1e-12 absolute of the oracle's
  (they are 1e-10 .. 1e-6 themselves).
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
U = 2.0 ** -53
DEV = "cuda:0"


@pytest.fixture(scope="module")
def g(genp_lib):
    import paper_1212_4560_gb300 as genp
    return genp


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("m,n,r,toep", [(64, 64, 1, False), (128, 128, 8, False), (256, 256, 32, False),
                                        (100, 70, 5, False), (64, 64, 8, True), (256, 256, 32, True),
                                        (300, 200, 128, False)])
def test_lowrank_vs_oracle(g, m, n, r, toep):
    rng = np.random.default_rng(m + n + r)
    if m == n:
        A, S, T, s = (t.numpy() for t in W.lowrank(n, min(r, n), seed=m + r))
    else:
        A = rng.standard_normal((m, n))
    kind = g.TOEPLITZ if toep else g.GAUSSIAN
    G, Q, R, AQ, st = g.lowrank(torch.as_tensor(A).to(DEV), r, kind=kind, seed=11, stream_id=2)
    assert int(host(st)[0]) == 0
    Gr = oracle.sketch_multiplier(m, r, seed=11, stream=2, toeplitz=toep)
    assert np.array_equal(host(G), Gr)
    ref = oracle.lowrank_approx(A, Gr)
    q = host(Q)
    kB = np.linalg.cond(ref["B"])
    assert np.linalg.norm(q.T @ q - np.eye(r), 2) <= 100 * n * r * U
    assert np.linalg.norm(q - ref["Q"], 2) <= 1e3 * n * r * U * kB
    Rm = host(R)
    assert np.allclose(np.tril(Rm, -1), 0.0, atol=1e3 * n * U * np.abs(Rm).max())
    assert np.all(np.diag(Rm) > 0)
    assert np.linalg.norm(host(AQ) - A @ q, 2) <= 1e3 * n * U * np.linalg.norm(A, 2)


@pytest.mark.parametrize("toep", [False, True])
def test_lowrank_table_residuals(g, toep):
    """The quantities of Tables 7.2 / 7.3 on their inputs (n = 128, q = 8):
    rn2 = ||A - A Q Q^T|| between sigma_{q+1} = 1e-10 and the oracle's value
    plus 1e-12; rn1 likewise."""
    n, q = 128, 8
    A, S, T, s = (t.numpy() for t in W.lowrank(n, q, seed=3))
    G, Q, R, AQ, st = g.lowrank(torch.as_tensor(A).to(DEV), q, kind=g.TOEPLITZ if toep else g.GAUSSIAN, seed=5)
    ref = oracle.lowrank_approx(A, oracle.sketch_multiplier(n, q, seed=5, toeplitz=toep))
    rn1, rn2 = oracle.lowrank_residuals(A, A.T @ host(G), host(Q), host(AQ), T[:, :q])
    r1, r2 = oracle.lowrank_residuals(A, ref["B"], ref["Q"], ref["AQ"], T[:, :q])
    assert rn2 >= 1e-10 * (1 - 1e-6)
    assert abs(rn2 - r2) <= 1e-12 and abs(rn1 - r1) <= 1e-12


def test_lowrank_exact_rank(g):
    n, q = 256, 32
    A, S, T, s = (t.numpy() for t in W.lowrank(n, q, seed=6))
    A = (S[:, :q] * s[:q]) @ T[:, :q].T
    G, Q, R, AQ, st = g.lowrank(torch.as_tensor(A).to(DEV), q, seed=1)
    q_ = host(Q)
    assert np.linalg.norm(A - host(AQ) @ q_.T, 2) <= 1e-13


def test_lowrank_rejects_bad_args(g):
    import ctypes
    lib = g._lib.load()
    A = torch.zeros((8, 8), dtype=torch.float64, device=DEV)
    Q = torch.zeros((8, 8), dtype=torch.float64, device=DEV)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    assert lib.genp_lowrank(8, 8, p(A), 8, 0, 0, 0, 0, None, 0, p(Q), 8, None, 0, None, 0, None, s) == -1   # r = 0
    assert lib.genp_lowrank(8, 8, p(A), 8, 9, 0, 0, 0, None, 0, p(Q), 8, None, 0, None, 0, None, s) == -1   # r > n
    assert lib.genp_lowrank(8, 8, p(A), 8, 2, 2, 0, 0, None, 0, p(Q), 8, None, 0, None, 0, None, s) == -1   # kind


# ------------------------------------------------ numerical rank (App. B)

@pytest.mark.parametrize("n,q,seed", [(64, 1, 0), (64, 8, 1), (128, 8, 2), (128, 32, 3), (256, 32, 4), (256, 17, 5)])
def test_numerical_rank_vs_oracle(g, n, q, seed):
    """Same rank as the oracle's search (exact kappa by SVD there, power and
    inverse iteration here: the inputs' gap, 1e4 against 1e9, leaves no
    decision near cond_max = 1e6), and the same basis A^T G_rank within the
    FP64 GEMM's 2 gamma_n |A|^T |G|."""
    A, S, T, s = (t.numpy() for t in W.lowrank(n, q, seed))
    r_hi = min(n, 128)
    rank, B = g.numerical_rank(torch.as_tensor(A).to(DEV), 0, r_hi, cond_max=1e6, seed=seed + 7)
    G = oracle.sketch_multiplier(n, r_hi, seed=seed + 7)
    rref, Bref, trace = oracle.numerical_rank(A, 0, r_hi, 1e6, G)
    assert rank == rref == q
    gam = 2 * n * U / (1 - 2 * n * U)
    assert np.all(np.abs(host(B) - Bref) <= gam * (np.abs(A).T @ np.abs(G[:, :q])))


def test_numerical_rank_ranges(g):
    A, S, T, s = (t.numpy() for t in W.lowrank(64, 8, 0))
    Ad = torch.as_tensor(A).to(DEV)
    assert g.numerical_rank(Ad, 5, 5, seed=1)[0] == 5
    assert g.numerical_rank(Ad, 0, 4, seed=1)[0] == 4
    assert g.numerical_rank(Ad, 12, 32, seed=1)[0] == 12
    assert g.numerical_rank(Ad, 0, 0, seed=1)[0] == 0


def test_cond_estimate_matches_svd(g):
    """COND's kappa estimate on a well separated full-rank sketch: the search
    over [r, r] performs no test, so test through a range whose midpoint is
    r: a matrix with kappa(A^T G_r) known from the SVD, cond_max just above
    and just below it (factor 2 either way)."""
    n, q = 128, 16
    A, S, T, s = (t.numpy() for t in W.lowrank(n, q, 2))
    G = oracle.sketch_multiplier(n, 16, seed=3)      # the sketch of width r_hi = 16
    kappa = np.linalg.cond(A.T @ G)
    Ad = torch.as_tensor(A).to(DEV)
    # range [15, 16]: the single test is at r = 16
    assert g.numerical_rank(Ad, 15, 16, cond_max=2 * kappa, seed=3)[0] == 16
    assert g.numerical_rank(Ad, 15, 16, cond_max=kappa / 2, seed=3)[0] == 15
