"""The left multiplier (C = G A, Cor. 4.1's GM half) on the GPU vs the CPU
oracle, through the C ABI.

Tolerances (u = 2^-53, gamma_k = k u / (1 - k u)):
* C = G A with a dense G in FP64: |dC| <= 2 gamma_n |G||A|; with the
  sparse +-1 G (exact signed gathers of at most 4 terms): bit-exact up to
  the order of a 4-term sum, |dC| <= 2 gamma_4 |G||A|; circulant / Toeplitz
  through the DFT, per column ||dc||_2 <= 8 log2(cn) u ||a||_2 ||G||_2;
* solve + refinement: eta <= 1e-14 and the GEPP solution within
  1e-14 kappa_inf(A), for classic refinement and GMRES-IR;
* adjoint: <= 1e-10 of the oracle gradient (GEPP on A^T).
"""
import ctypes
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
U = 2.0 ** -53
DEV = "cuda:0"


def gamma(k):
    return k * U / (1 - k * U)


@pytest.fixture(scope="module")
def g(genp_lib):
    import paper_1212_4560_gb300 as genp
    return genp


def cu(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dtype)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def test_side_setting(g, genp_lib):
    G = g.make_multiplier(g.GAUSSIAN, 8, seed=1)
    assert genp_lib.genp_multiplier_side(G.handle, -1) == 0
    assert genp_lib.genp_multiplier_side(G.handle, 1) == 0
    assert genp_lib.genp_multiplier_side(G.handle, -1) == 1
    assert genp_lib.genp_multiplier_side(G.handle, 2) == -1
    assert genp_lib.genp_multiplier_side(None, 0) == -1


@pytest.mark.parametrize("kind,n", [(0, 1), (0, 130), (1, 256), (1, 100), (2, 200), (5, 128), (5, 90), (6, 64)])
def test_precondition_left(g, kind, n):
    rng = np.random.default_rng(kind * 100 + n)
    A = rng.standard_normal((n, n))
    G = g.make_multiplier(kind, n, seed=7, side=g.LEFT)
    C = torch.empty((n, n), dtype=torch.float64, device=DEV)
    g.precondition(G, cu(A), C)
    M = oracle.multiplier(kind, n, seed=7)
    ref = oracle.precondition_left(A, M)
    d = host(C) - ref
    fft = kind in (1, 5) and (n & (n - 1)) == 0
    if fft:
        col = M["g"] if kind == 1 else None
        if kind == 5:
            col = np.zeros(2 * n)
            for dd in range(-(n - 1), n):
                col[dd % (2 * n)] = M["t"][dd + n - 1]
        gnorm = np.abs(np.fft.fft(col)).max()
        bound = 8 * math.log2(len(col)) * U * np.linalg.norm(A, axis=0) * gnorm
        assert np.all(np.linalg.norm(d, axis=0) <= bound)
    else:
        assert np.all(np.abs(d) <= 4 * gamma(n + 2) * (np.abs(M["G"]) @ np.abs(A)))


@pytest.mark.parametrize("kind", [0, 1, 2, 5])
def test_left_end_to_end(g, kind):
    """The rank-16 workload: GENP of G A is safe, x = U^-1 L^-1 G b refined
    to eta <= 1e-14, equal to the GEPP solution within 1e-14 kappa and to
    the oracle's left-multiplier solution."""
    A, _, B = (t.numpy() for t in W.lead_deficient(256, 32, 16, 2, seed=3))
    X, info, G, F = g.solve_system(cu(A), cu(B), kind=kind, seed=5, refine_steps=8, tol=1e-16, side=g.LEFT)
    x = host(X)
    assert info.breakdown_step == -1
    assert oracle.backward_error(A, x, B) <= 1e-14
    kappa = np.linalg.cond(A, np.inf)
    xd = oracle.gepp_solve(A, B)
    assert np.abs(x - xd).max() / np.abs(xd).max() <= 1e-14 * kappa
    ref = oracle.solve(A, B, oracle.multiplier(kind, 256, seed=5), refine_steps=8, tol=1e-16, side="left")
    assert np.abs(x - ref["x"]).max() / np.abs(ref["x"]).max() <= 1e-14 * kappa
    # the unrefined solution: x0 = U^-1 L^-1 (G b) of the oracle's factors, within the factors' conditioning
    X0 = torch.empty_like(cu(B))
    g.solve(F, G, cu(B), X0)
    r0 = oracle.solve(A, B, oracle.multiplier(kind, 256, seed=5), refine_steps=0, side="left")
    kc = np.linalg.cond(r0["C"], np.inf)
    assert np.abs(host(X0) - r0["x"]).max() <= 1e-13 * kc * max(1.0, np.abs(r0["x"]).max())


@pytest.mark.parametrize("prec,kind", [("FP32", 0), ("FP32", 1), ("BF16_SLICED", 0), ("FP64", 2)])
def test_left_gmres_ir(g, prec, kind):
    n = 300
    A, _, B = (t.numpy() for t in W.lead_deficient(n, 32, 16, 3, seed=9))
    X, info, G, F = g.solve_system(cu(A), cu(B), kind=kind, seed=2, prec=getattr(g, prec), refine_steps=8,
                                   tol=1e-16, method=1, side=g.LEFT)
    x = host(X)
    assert oracle.backward_error(A, x, B) <= 1e-14
    xd = oracle.gepp_solve(A, B)
    assert np.abs(x - xd).max() <= 1e-14 * np.linalg.cond(A, np.inf) * np.abs(xd).max()
    assert g._lib.load().genp_device_check(1) == 0


def test_left_unsupported_precisions(g):
    n = 64
    G = g.make_multiplier(g.GAUSSIAN, n, seed=1, value_grid=g.BF16, side=g.LEFT)
    A = torch.zeros((n, n), dtype=torch.float64, device=DEV)
    C = torch.empty((n, n), dtype=torch.float32, device=DEV)
    st = g._lib.load().genp_precondition(G.handle, ctypes.c_void_p(A.data_ptr()), n, g.FP64,
                                         ctypes.c_void_p(C.data_ptr()), n, g.BF16,
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == -7     # GENP_ERR_UNSUPPORTED


@pytest.mark.parametrize("kind", [0, 1, 5, 6])
def test_left_adjoint(g, kind):
    """Lambda = A^{-T} gX = G^T z with z = C^{-T} gX = G^{-T} Lambda from the
    left factors, against the oracle's gradient (GEPP on A^T).  z is as
    accurate as a solve with C (relative error up to about n kappa(C) u) but
    is larger than Lambda by up to ||G^{-1}||, and G^T brings that error back
    at ||G||: relative error <= n kappa(G) kappa(C) u, a factor kappa(G) above
    the right multiplier's bound (1e-10 there; the right-side test)."""
    n, nrhs = 64, 3
    A, _, B = (t.numpy() for t in W.shifted(1, n, nrhs, seed=7))
    A, B = A[0], B[0]
    X, info, G, F = g.solve_system(cu(A), cu(B), kind=kind, seed=3, refine_steps=5, tol=1e-17, side=g.LEFT)
    x = host(X)
    dA = torch.empty((n, n), dtype=torch.float64, device=DEV)
    dB = torch.empty((n, nrhs), dtype=torch.float64, device=DEV)
    g.adjoint(F, G, cu(2.0 * x), X, dA, dB)
    dA_ref, dB_ref = oracle.adjoint(A, x, 2.0 * x)
    M = oracle.multiplier(kind, n, seed=3)
    tol = max(1e-10, n * np.linalg.cond(M["G"]) * np.linalg.cond(oracle.precondition_left(A, M)) * U)
    assert np.linalg.norm(host(dA) - dA_ref) <= tol * np.linalg.norm(dA_ref)
    assert np.linalg.norm(host(dB) - dB_ref) <= tol * np.linalg.norm(dB_ref)
