"""The Gaussian Toeplitz (Definition 3.2) and +-1 Householder multipliers
on the GPU vs the CPU oracle, through the C ABI.

Tolerances (u = 2^-53, gamma_k = k u / (1 - k u)):
* multiplier entries: bit-exact (same Philox counters, same polar method;
  the Householder entries 1 - (2 u_i u_j)/n in the same operation order);
* Toeplitz C = A T through the DFT of its circulant embedding of order 2n:
  per row ||dc||_2 <= 8 log2(2n) u ||a||_2 ||G_2n||_2, ||G_2n||_2 the largest
  |DFT| of the embedding's first column (the FFT error of the length-2n
  correlation of the zero-padded row); by the direct product (n not a power
  of two): |dC| <= 2 gamma_n |A||T|;
* Householder C = A - (2/n)(A u) u^T: |dC| <= 4 gamma_{n+2} |A||H| (the dot
  product's gamma_n sum_i |a_i| (2/n) is below gamma_n (|A||H|) for n >= 4,
  plus the roundings of 2/n, the product and the update);
* solve + refinement: eta <= 1e-14 and forward error <= 1e-14 kappa_inf(A);
* adjoint: <= 1e-10 of the oracle gradient (GEPP on A^T).
"""
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


def embedding(t, n):
    """First column of the circulant of order 2n whose leading n x n block is
    the Toeplitz matrix with entries t_{-(n-1)} .. t_{n-1}."""
    e = np.zeros(2 * n)
    for d in range(-(n - 1), n):
        e[d % (2 * n)] = t[d + n - 1]
    return e


@pytest.mark.parametrize("n", [1, 2, 5, 100, 1024, 4096])
def test_toeplitz_multiplier_bit_exact(g, n):
    G = g.make_multiplier(g.TOEPLITZ, n, seed=21, stream_id=2)
    col = torch.empty(2 * n, dtype=torch.float64, device=DEV)
    g.multiplier_export(G, first_col=col)
    ref = oracle.multiplier(5, n, seed=21, stream=2)
    assert np.array_equal(host(col), embedding(ref["t"], n))
    if n <= 1024:
        D = torch.empty((n, n), dtype=torch.float64, device=DEV)
        g.multiplier_export(G, dense=D)
        assert np.array_equal(host(D), ref["G"])
    kind = __import__("ctypes").c_int()
    g._lib.load().genp_multiplier_query(G.handle, None, __import__("ctypes").byref(kind), None)
    assert kind.value == g.TOEPLITZ


def test_toeplitz_fp32_grid_and_redraw(g):
    n = 300
    G = g.make_multiplier(g.TOEPLITZ, n, seed=4, value_grid=g.FP32)
    col = torch.empty(2 * n, dtype=torch.float64, device=DEV)
    g.multiplier_export(G, first_col=col)
    assert np.array_equal(host(col), embedding(oracle.multiplier(5, n, seed=4, grid="fp32")["t"], n))
    g.redraw_multiplier(G, seed=9, stream_id=1)
    g.multiplier_export(G, first_col=col)
    assert np.array_equal(host(col), embedding(oracle.multiplier(5, n, seed=9, stream=1, grid="fp32")["t"], n))


@pytest.mark.parametrize("n", [1, 2, 3, 64, 100, 256])
def test_householder_multiplier_bit_exact(g, n):
    G = g.make_multiplier(g.HOUSEHOLDER_PM1, n, seed=33)
    u = torch.empty(n, dtype=torch.float64, device=DEV)
    D = torch.empty((n, n), dtype=torch.float64, device=DEV)
    g.multiplier_export(G, dense=D, first_col=u)
    ref = oracle.multiplier(6, n, seed=33)
    assert np.array_equal(host(u), ref["u"])
    assert np.array_equal(host(D), ref["G"])


@pytest.mark.parametrize("n", [2, 64, 256, 1024, 4096, 100, 37])
def test_precondition_toeplitz(g, n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    G = g.make_multiplier(g.TOEPLITZ, n, seed=3)
    C = torch.empty((n, n), dtype=torch.float64, device=DEV)
    g.precondition(G, cu(A), C)
    M = oracle.multiplier(5, n, seed=3)
    ref = oracle.precondition(A, M)
    d = host(C) - ref
    if (n & (n - 1)) == 0:          # DFT of the order-2n embedding
        gnorm = np.abs(np.fft.fft(embedding(M["t"], n))).max()
        bound = 8 * math.log2(2 * n) * U * np.linalg.norm(A, axis=1) * gnorm
        assert np.all(np.linalg.norm(d, axis=1) <= bound)
    else:                           # direct product
        assert np.all(np.abs(d) <= 2 * gamma(n) * (np.abs(A) @ np.abs(M["G"])))


@pytest.mark.parametrize("n", [4, 64, 100, 256, 1000])
def test_precondition_householder(g, n):
    rng = np.random.default_rng(n + 1)
    A = rng.standard_normal((n, n))
    G = g.make_multiplier(g.HOUSEHOLDER_PM1, n, seed=8)
    C = torch.empty((n, n), dtype=torch.float64, device=DEV)
    g.precondition(G, cu(A), C)
    M = oracle.multiplier(6, n, seed=8)
    ref = oracle.precondition(A, M)
    assert np.all(np.abs(host(C) - ref) <= 4 * gamma(n + 2) * (np.abs(A) @ np.abs(M["G"])))
    # FP32 storage of C: the same product rounded once more
    C32 = torch.empty((n, n), dtype=torch.float32, device=DEV)
    g.precondition(G, cu(A), C32, c_prec=g.FP32)
    assert np.all(np.abs(host(C32).astype(np.float64) - ref)
                  <= 4 * gamma(n + 2) * (np.abs(A) @ np.abs(M["G"])) + 2.0 ** -24 * np.abs(ref))


@pytest.mark.parametrize("n,nrhs,trans", [(64, 1, False), (64, 3, True), (100, 16, False), (1000, 2, True)])
def test_apply_multipliers(g, n, nrhs, trans):
    """x = G y and x = G^T y (the solve and the adjoint) for both kinds,
    through genp_solve with identity factors: C = I makes X = G B."""
    rng = np.random.default_rng(n * nrhs)
    Y = rng.standard_normal((n, nrhs))
    for kind in (5, 6):
        M = oracle.multiplier(kind, n, seed=12)
        ref = oracle.apply_multiplier(M, Y, trans=trans)
        G = g.make_multiplier(kind, n, seed=12)
        I = torch.eye(n, dtype=torch.float64, device=DEV)
        F = g.factor(I)
        X = torch.empty((n, nrhs), dtype=torch.float64, device=DEV)
        if trans:     # dB of the adjoint with X = 0 is lambda = L^-T U^-T G^T gX = G^T gX
            dB = torch.empty((n, nrhs), dtype=torch.float64, device=DEV)
            g.adjoint(F, G, cu(Y), torch.zeros((n, nrhs), dtype=torch.float64, device=DEV), None, dB)
            got = host(dB)
        else:
            g.solve(F, G, cu(Y), X)
            got = host(X)
        bound = 4 * gamma(n + 2) * (np.abs(M["G"].T if trans else M["G"]) @ np.abs(Y))
        if kind == 5 and (n & (n - 1)) == 0:
            gnorm = np.abs(np.fft.fft(embedding(M["t"], n))).max()
            bound = 8 * math.log2(2 * n) * U * np.linalg.norm(Y, axis=0) * gnorm
            assert np.all(np.linalg.norm(got - ref, axis=0) <= bound)
        else:
            assert np.all(np.abs(got - ref) <= bound)


@pytest.mark.parametrize("n", [256, 300])
def test_toeplitz_end_to_end(g, n):
    """Leading 32 x 32 block of rank 16: the Toeplitz multiplier makes GENP
    safe (DFT path at n = 256, direct at n = 300); refinement reaches
    eta <= 1e-14 and the GEPP solution within 1e-14 kappa."""
    A, _, B = (t.numpy() for t in W.lead_deficient(n, 32, 16, 2, seed=1))
    X, info, G, F = g.solve_system(cu(A), cu(B), kind=g.TOEPLITZ, seed=6, refine_steps=8, tol=1e-16)
    x = host(X)
    assert info.breakdown_step == -1
    assert oracle.backward_error(A, x, B) <= 1e-14
    xd = oracle.gepp_solve(A, B)
    assert np.abs(x - xd).max() / np.abs(xd).max() <= 1e-14 * np.linalg.cond(A, np.inf)
    ref = oracle.solve(A, B, oracle.multiplier(5, n, seed=6), refine_steps=8, tol=1e-16)
    assert np.abs(x - ref["x"]).max() / np.abs(ref["x"]).max() <= 1e-14 * np.linalg.cond(A, np.inf)


def test_householder_end_to_end(g):
    """Paper-shaped inputs (n/2 x n/2 leading block of numerical rank
    n/2 - 1): the reflector, a rank-one change, repairs GENP; refinement
    reaches eta <= 1e-14."""
    n = 256
    A, _, B = (t.numpy() for t in W.table71(n, 2))
    X, info, G, F = g.solve_system(cu(A), cu(B), kind=g.HOUSEHOLDER_PM1, seed=6, refine_steps=8, tol=1e-16)
    x = host(X)
    assert oracle.backward_error(A, x, B) <= 1e-14
    xd = oracle.gepp_solve(A, B)
    assert np.abs(x - xd).max() / np.abs(xd).max() <= 1e-14 * np.linalg.cond(A, np.inf)


@pytest.mark.parametrize("prec", ["FP32", "BF16_SLICED"])
def test_toeplitz_gmres_ir(g, prec):
    n = 512
    A, _, B = (t.numpy() for t in W.lead_deficient(n, 32, 16, 1, seed=2))
    X, info, G, F = g.solve_system(cu(A), cu(B), kind=g.TOEPLITZ, seed=8, prec=getattr(g, prec), refine_steps=8,
                                   tol=1e-16, method=1)
    x = host(X)
    assert oracle.backward_error(A, x, B) <= 1e-14
    assert g._lib.load().genp_device_check(1) == 0


@pytest.mark.parametrize("kind", [5, 6])
def test_adjoint_new_multipliers(g, kind):
    n, nrhs = 64, 3
    A, _, B = (t.numpy() for t in W.shifted(1, n, nrhs, seed=7))
    A, B = A[0], B[0]
    X, info, G, F = g.solve_system(cu(A), cu(B), kind=kind, seed=3, refine_steps=5, tol=1e-17)
    x = host(X)
    dA = torch.empty((n, n), dtype=torch.float64, device=DEV)
    dB = torch.empty((n, nrhs), dtype=torch.float64, device=DEV)
    g.adjoint(F, G, cu(2.0 * x), X, dA, dB)
    dA_ref, dB_ref = oracle.adjoint(A, x, 2.0 * x)
    assert np.linalg.norm(host(dA) - dA_ref) <= 1e-10 * np.linalg.norm(dA_ref)
    assert np.linalg.norm(host(dB) - dB_ref) <= 1e-10 * np.linalg.norm(dB_ref)
