"""GPU path vs the CPU oracle, element by element, through the C ABI.

Tolerances (u = 2^-53, gamma_k = k u / (1 - k u)):
* random-number work (multiplier entries, sparse indices and signs): bit-exact;
* products of integer-valued data and the +-1 sparse gather: bit-exact;
* dense C = A G in FP64: |dC| <= 2 gamma_n |A||G| (each side within gamma_n
  of the exact product, any summation order, with or without FMA);
* circulant C = A G by FFT: per row ||dc||_2 <= 8 log2(n) u ||a||_2 ||G||_2
  (normwise FFT error bound; ||G||_2 = max_k |DFT(g)_k| for a circulant);
* GENP factors: backward error |L U - C| <= 3 gamma_n |L||U| (Higham,
  Thm. 9.3, plus the rounding of the check itself); pinned exactly on
  integer L0 U0 inputs;
* solve + refinement: normwise backward error <= 1e-14 and forward error
  <= 1e-14 kappa_inf(A) against the FP64 oracle, as the method targets.
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


# ---------------------------------------------------------------- multipliers

@pytest.mark.parametrize("n", [1, 2, 17, 64, 257])
def test_dense_multiplier_bit_exact(g, n):
    G = g.make_multiplier(g.GAUSSIAN, n, seed=12345, stream_id=3)
    D = torch.empty((n, n), dtype=torch.float64, device=DEV)
    g.multiplier_export(G, dense=D)
    ref = oracle.multiplier(0, n, seed=12345, stream=3)["G"]
    assert np.array_equal(host(D), ref)


@pytest.mark.parametrize("n", [1, 5, 100, 1024, 8192])
def test_circulant_multiplier_bit_exact(g, n):
    G = g.make_multiplier(g.CIRCULANT, n, seed=7)
    col = torch.empty(n, dtype=torch.float64, device=DEV)
    g.multiplier_export(G, first_col=col)
    ref = oracle.multiplier(1, n, seed=7)
    assert np.array_equal(host(col), ref["g"])
    if n <= 1024:
        D = torch.empty((n, n), dtype=torch.float64, device=DEV)
        g.multiplier_export(G, dense=D)
        assert np.array_equal(host(D), ref["G"])


@pytest.mark.parametrize("n,nnz", [(1, 4), (3, 4), (100, 4), (1000, 2), (8192, 4)])
def test_sparse_multiplier_bit_exact(g, n, nnz):
    G = g.make_multiplier(g.SPARSE_PM1, n, seed=99, nnz_per_col=nnz)
    rows = torch.empty((nnz, n), dtype=torch.int32, device=DEV)
    signs = torch.empty((nnz, n), dtype=torch.int8, device=DEV)
    g.multiplier_export(G, rows=rows, signs=signs)
    ref = oracle.multiplier(2, n, seed=99, nnz=nnz)
    assert np.array_equal(host(rows), ref["rows"])
    assert np.array_equal(host(signs), ref["signs"])
    if n <= 1000:
        D = torch.empty((n, n), dtype=torch.float64, device=DEV)
        g.multiplier_export(G, dense=D)
        assert np.array_equal(host(D), ref["G"])


def test_bf16_and_fp32_grids(g):
    n = 96
    G = g.make_multiplier(g.GAUSSIAN, n, seed=5, value_grid=g.BF16)
    D = torch.empty((n, n), dtype=torch.float64, device=DEV)
    g.multiplier_export(G, dense=D)
    d = host(D)
    assert np.array_equal(torch.tensor(d).to(torch.bfloat16).double().numpy(), d)   # on the BF16 grid
    raw = oracle.multiplier(0, n, seed=5)["G"]
    # nearest BF16 value of the drawn entry (ties-to-even; torch rounds FP64 -> BF16 directly)
    assert np.array_equal(torch.tensor(raw).to(torch.bfloat16).double().numpy(), d)
    # FP32 grid: drawn by the polar method in single precision, bit-exact
    G32 = g.make_multiplier(g.GAUSSIAN, n, seed=5, value_grid=g.FP32)
    g.multiplier_export(G32, dense=D)
    assert np.array_equal(host(D), oracle.multiplier(0, n, seed=5, grid="fp32")["G"])
    C32 = g.make_multiplier(g.CIRCULANT, 1000, seed=6, value_grid=g.FP32)
    col = torch.empty(1000, dtype=torch.float64, device=DEV)
    g.multiplier_export(C32, first_col=col)
    assert np.array_equal(host(col), oracle.multiplier(1, 1000, seed=6, grid="fp32")["g"])


# ---------------------------------------------------------------- C = A G

@pytest.mark.parametrize("n", [1, 3, 33, 130, 256])
def test_precondition_dense(g, n):
    A, _, _ = W.lead_deficient(n, min(8, n), min(4, n), 1, seed=n)
    A = A.numpy()
    G = g.make_multiplier(g.GAUSSIAN, n, seed=1)
    C = torch.empty((n, n), dtype=torch.float64, device=DEV)
    g.precondition(G, cu(A), C)
    Gm = oracle.multiplier(0, n, seed=1)["G"]
    ref = oracle.precondition(A, {"kind": 0, "n": n, "G": Gm})
    assert np.all(np.abs(host(C) - ref) <= 2 * gamma(n) * (np.abs(A) @ np.abs(Gm)))


def test_precondition_dense_ld_padding(g):
    """Leading dimensions larger than n on every operand."""
    n = 70
    A = np.random.default_rng(0).standard_normal((n, n))
    Ap = torch.zeros((n, n + 9), dtype=torch.float64, device=DEV)
    Ap[:, :n] = cu(A)
    Cp = torch.full((n, n + 5), 7.0, dtype=torch.float64, device=DEV)
    G = g.make_multiplier(g.GAUSSIAN, n, seed=2)
    g.precondition(G, Ap[:, :n], Cp[:, :n])
    Gm = oracle.multiplier(0, n, seed=2)["G"]
    c = host(Cp)
    assert np.all(c[:, n:] == 7.0)                         # padding untouched
    assert np.all(np.abs(c[:, :n] - A @ Gm) <= 2 * gamma(n) * (np.abs(A) @ np.abs(Gm)))


@pytest.mark.parametrize("n", [2, 64, 256, 1024, 100, 37])
def test_precondition_circulant(g, n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    G = g.make_multiplier(g.CIRCULANT, n, seed=3)
    C = torch.empty((n, n), dtype=torch.float64, device=DEV)
    g.precondition(G, cu(A), C)
    M = oracle.multiplier(1, n, seed=3)
    ref = oracle.precondition(A, M)
    d = host(C) - ref
    if (n & (n - 1)) == 0:          # FFT path
        gnorm = np.abs(np.fft.fft(M["g"])).max()
        bound = 8 * max(1, math.log2(n)) * U * np.linalg.norm(A, axis=1) * gnorm
        assert np.all(np.linalg.norm(d, axis=1) <= bound)
    else:                           # direct product
        assert np.all(np.abs(d) <= 2 * gamma(n) * (np.abs(A) @ np.abs(M["G"])))


@pytest.mark.parametrize("n", [1, 5, 200, 1000])
def test_precondition_sparse_bit_exact(g, n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    G = g.make_multiplier(g.SPARSE_PM1, n, seed=4)
    C = torch.empty((n, n), dtype=torch.float64, device=DEV)
    g.precondition(G, cu(A), C)
    ref = oracle.precondition(A, oracle.multiplier(2, n, seed=4))
    assert np.array_equal(host(C), ref)


# ---------------------------------------------------------------- GENP

def _integer_LU(n, rng):
    L0 = np.tril(rng.integers(-2, 3, (n, n)), -1) + np.eye(n, dtype=np.int64)
    U0 = np.triu(rng.integers(-2, 3, (n, n)), 1) + np.diag(rng.choice([-1, 1], n))
    return L0, U0


@pytest.mark.parametrize("n", [1, 2, 17, 64, 65, 130, 200])
def test_factor_integer_exact(g, n):
    """C = L0 U0 with small-integer factors: all intermediates are exact, the
    pivot-free LU is unique, so the GPU must return L0 and U0 bit for bit."""
    rng = np.random.default_rng(1000 + n)
    L0, U0 = _integer_LU(n, rng)
    C0 = L0 @ U0
    if np.abs(C0).max() >= 2**50:
        pytest.skip("entries too large for exactness")
    C = cu(C0.astype(float))
    F = g.factor(C)
    info = g.info_fetch(F)
    assert info.breakdown_step == -1
    LU = host(C)
    L, Uf = oracle.split_lu(LU)
    assert np.array_equal(L, L0.astype(float))
    assert np.array_equal(Uf, U0.astype(float))
    assert info.min_abs_pivot == 1.0 and info.max_abs_pivot == 1.0


@pytest.mark.parametrize("n,nb", [(3, 0), (31, 0), (63, 0), (129, 0), (256, 0), (256, 32), (200, 128), (97, 1)])
def test_factor_vs_oracle(g, n, nb):
    A, _, _ = W.lead_deficient(n, min(16, n), min(8, n), 1, seed=n)
    M = oracle.multiplier(0, n, seed=9)
    C0 = oracle.precondition(A.numpy(), M)
    C = cu(C0)
    F = g.factor(C, nb=nb)
    info = g.info_fetch(F)
    assert info.breakdown_step == -1
    LU = host(C)
    L, Uf = oracle.split_lu(LU)
    assert np.all(np.abs(L @ Uf - C0) <= 3 * gamma(n) * (np.abs(L) @ np.abs(Uf)) + 1e-300)
    LUo, k = oracle.genp(C0)
    assert k == -1
    assert np.linalg.norm(LU - LUo) <= 1e-9 * np.linalg.norm(LUo)
    piv = np.abs(np.diag(LUo))
    assert info.min_abs_pivot == pytest.approx(piv.min(), rel=1e-9)
    assert info.max_abs_pivot == pytest.approx(piv.max(), rel=1e-9)
    growth = np.abs(np.triu(LUo)).max() / np.abs(C0).max()
    assert info.growth == pytest.approx(growth, rel=1e-9)


def test_breakdown_reported(g):
    """[[0,1],[1,0]]: GENP meets a zero pivot at step 0; a zero pivot planted
    at step 70 (second block) is reported as step 70."""
    C = cu(np.array([[0.0, 1.0], [1.0, 0.0]]))
    F = g.factor(C)
    info = g.info_fetch(F)
    assert info.breakdown_step == 0
    assert info.status == -2                                # GENP_ERR_BREAKDOWN
    n = 100
    rng = np.random.default_rng(3)
    L0, U0 = _integer_LU(n, rng)
    U0[70, 70] = 0
    F2 = g.factor(cu((L0 @ U0).astype(float)))
    assert g.info_fetch(F2).breakdown_step == 70


# ---------------------------------------------------------------- solve / refine

@pytest.mark.parametrize("kind", [0, 1, 2])
def test_cfg_n256_end_to_end(g, kind):
    """The n=256 workload (leading 32x32 block of rank 16, one RHS): GPU
    solve + refinement reaches backward error <= 1e-14 and agrees with the
    oracle's solution within 1e-14 kappa."""
    A, Xs, B = (t.numpy() for t in W.lead_deficient(256, 32, 16, 1, seed=0))
    X, info, G, F = g.solve_system(cu(A), cu(B), kind=kind, seed=5, refine_steps=8, tol=1e-16)
    x = host(X)
    eta = oracle.backward_error(A, x, B)
    assert eta <= 1e-14
    # the device's own backward error: each side's residual is exact to within
    # gamma_{n+1} (|A||x| + |b|), so the two values of eta agree to 2 gamma_{n+1}
    assert info.bwd_err[-1] <= 1e-14
    assert abs(info.bwd_err[-1] - eta) <= 2 * gamma(257)
    kappa = np.linalg.cond(A, np.inf)
    xd = oracle.gepp_solve(A, B)
    assert np.abs(x - xd).max() / np.abs(xd).max() <= 1e-14 * kappa
    ref = oracle.solve(A, B, oracle.multiplier(kind, 256, seed=5), refine_steps=8, tol=1e-16)
    assert np.abs(x - ref["x"]).max() / np.abs(ref["x"]).max() <= 1e-14 * kappa


@pytest.mark.parametrize("n,nrhs,kind", [(1, 1, 0), (2, 3, 0), (17, 2, 1), (33, 16, 2), (65, 5, 0), (128, 16, 1),
                                          (300, 4, 2)])
def test_solve_shapes(g, n, nrhs, kind):
    A, _, B = (t.numpy() for t in W.lead_deficient(n, min(8, n), min(4, n), nrhs, seed=n + nrhs))
    X, info, G, F = g.solve_system(cu(A), cu(B), kind=kind, seed=11, refine_steps=10, tol=1e-16)
    x = host(X)
    assert oracle.backward_error(A, x, B) <= 1e-14
    # unrefined solution agrees with the oracle's unrefined method solution
    X0 = torch.empty_like(cu(B))
    g.solve(F, G, cu(B), X0)
    M = oracle.multiplier(kind, n, seed=11)
    r = oracle.solve(A, B, M, refine_steps=0)
    kappa_c = np.linalg.cond(r["C"], np.inf)
    assert np.abs(host(X0) - r["x"]).max() <= 1e-13 * kappa_c * max(1.0, np.abs(r["x"]).max())


@pytest.mark.parametrize("prec", ["FP64", "FP32"])
@pytest.mark.parametrize("n,nrhs", [(1100, 1), (1100, 5), (2113, 16), (1500, 19), (64, 2), (129, 1)])
def test_triangular_solves_streaming(g, prec, n, nrhs):
    """The persistent triangular solves (several work items per block column
    from n > 17 * 64 on, ragged last block, two right-hand-side chunks at
    nrhs > 16), forward and transposed, against the oracle's substitutions
    with the same factors.  C is diagonally dominant, so L and U are well
    conditioned and the forward error stays within a few n u |y|."""
    rng = np.random.default_rng(n + nrhs)
    C0 = rng.standard_normal((n, n)) / np.sqrt(n) + 4.0 * np.eye(n)
    dt = torch.float64 if prec == "FP64" else torch.float32
    u = 2.0 ** -53 if prec == "FP64" else 2.0 ** -24
    C = cu(C0, dt)
    F = g.factor(C, prec=getattr(g, prec))
    LU = host(C).astype(np.float64)
    G = g.make_multiplier(g.SPARSE_PM1, n, seed=3)
    Gd = torch.empty((n, n), dtype=torch.float64, device=DEV)
    g.multiplier_export(G, dense=Gd)
    Gm = host(Gd)
    B = rng.standard_normal((n, nrhs))
    X = torch.empty((n, nrhs), dtype=torch.float64, device=DEV)
    g.solve(F, G, cu(B), X)
    Bq = B.astype(np.float32).astype(np.float64) if prec == "FP32" else B
    y = oracle.lu_solve(LU, Bq)
    tol = 8 * n * u * (np.abs(Gm) @ np.abs(y)).max()
    assert np.abs(host(X) - Gm @ y).max() <= tol
    # transposed pair through the adjoint: dB = L^-T U^-T G^T gX
    gX = rng.standard_normal((n, nrhs))
    dB = torch.empty((n, nrhs), dtype=torch.float64, device=DEV)
    g.adjoint(F, G, cu(gX), X, None, dB)
    rhs = Gm.T @ gX
    if prec == "FP32":
        rhs = rhs.astype(np.float32).astype(np.float64)
    lam = oracle.lu_solve_T(LU, rhs)
    assert np.abs(host(dB) - lam).max() <= 8 * n * u * np.abs(lam).max()
    assert g._lib.load().genp_device_check(1) == 0


@pytest.mark.parametrize("prec,kind,nrhs", [("FP64", 0, 1), ("FP32", 1, 3), ("BF16X3", 0, 16), ("BF16X3", 2, 2)])
def test_gmres_ir(g, prec, kind, nrhs):
    """GMRES-IR (method 1): every precision of factors reaches eta <= 1e-14,
    each right-hand side in its own Krylov space; the result agrees with the
    definition-level GEPP solution within the forward-error bound."""
    n = 300
    A, _, B = (t.numpy() for t in W.lead_deficient(n, 32, 16, nrhs, seed=7))
    X, info, G, F = g.solve_system(cu(A), cu(B), kind=kind, seed=3, prec=getattr(g, prec), refine_steps=8,
                                   tol=1e-16, method=1)
    x = host(X)
    assert oracle.backward_error(A, x, B) <= 1e-14
    xr = oracle.gepp_solve(A, B)
    kappa = np.linalg.cond(A, np.inf)
    assert np.abs(x - xr).max() <= 1e-14 * kappa * np.abs(xr).max()
    assert len(info.bwd_err) == info.refine_iters + 1
    assert g._lib.load().genp_device_check(1) == 0


@pytest.mark.parametrize("n,seed", [(64, 0), (64, 5), (256, 7), (1024, 1), (1000, 2), (3000, 4)])
def test_circulant_pm1_bit_exact(g, n, seed):
    """The +-1 circulant draw (attempts included) equals the oracle's bit for bit."""
    G = g.make_multiplier(g.CIRCULANT_PM1, n, seed=seed)
    first = torch.empty(n, dtype=torch.float64, device=DEV)
    g.multiplier_export(G, first_col=first)
    M = oracle.multiplier(oracle.KIND_CIRCULANT_PM1, n, seed=seed)
    assert np.array_equal(host(first), M["g"])
    k = ctypes.c_int()
    g._lib.load().genp_multiplier_query(G.handle, None, ctypes.byref(k), None)
    assert k.value == g.CIRCULANT_PM1


@pytest.mark.parametrize("n", [64, 256, 1024])
def test_circulant_pm1_solves_table71_system(g, n):
    """The paper's test multiplier on the paper-shaped Table 7.1 system: one
    refinement step reaches the paper's residual level; plain GENP (the
    identity multiplier) does not."""
    A, _, B = (t.numpy() for t in W.table71(n, seed=3))
    X, info, G, F = g.solve_system(cu(A), cu(B), kind=g.CIRCULANT_PM1, seed=3, refine_steps=1, tol=0.0)
    x = host(X)
    res = np.linalg.norm(A @ x - B) / np.linalg.norm(B)
    assert res <= 1e-12
    Xp, infop, _, _ = g.solve_system(cu(A), cu(B), kind=g.IDENTITY, seed=0, refine_steps=0)
    resp = np.linalg.norm(A @ host(Xp) - B) / np.linalg.norm(B)
    assert resp > 1e3 * res


def test_identity_multiplier_breaks_down(g):
    A = np.array([[0.0, 1.0], [1.0, 0.0]])
    C = cu(A)
    G = g.make_multiplier(g.IDENTITY, 2, seed=0)
    g.precondition(G, cu(A), C)
    F = g.factor(C)
    assert g.info_fetch(F).breakdown_step == 0


def test_2x2_antidiagonal_solved(g):
    A = np.array([[0.0, 1.0], [1.0, 0.0]])
    B = np.array([[2.0], [3.0]])
    X, info, _, _ = g.solve_system(cu(A), cu(B), kind=g.GAUSSIAN, seed=4, refine_steps=3, tol=1e-16)
    assert np.allclose(host(X), [[3.0], [2.0]], rtol=0, atol=1e-15)
    assert info.breakdown_step == -1


def test_refinement_reports_history(g):
    n = 128
    A, _, B = (t.numpy() for t in W.lead_deficient(n, 16, 8, 2, seed=2))
    X, info, _, _ = g.solve_system(cu(A), cu(B), seed=1, refine_steps=6, tol=0.0)
    assert len(info.bwd_err) == info.refine_iters + 1
    assert info.bwd_err[-1] <= 1e-14
    # stops on stagnation (tol 0 cannot be met): the last step failed to halve eta
    assert info.bwd_err[-1] > 0.5 * info.bwd_err[-2] or info.refine_iters == 6


# ---------------------------------------------------------------- FP32 path

@pytest.mark.parametrize("kind,method", [(0, 1), (1, 0), (2, 0), (1, 1), (2, 1)])
def test_fp32_factor_with_fp64_refinement(g, kind, method):
    """FP32 factors, FP64 refinement, eta <= 1e-14 for every multiplier.
    Classic refinement (method 0) contracts by u32 kappa(C) growth per step;
    with the dense Gaussian multiplier (kappa(G) ~ 3n) that ratio nears 1/2
    and the stop rule (eta must halve) can end it just above 1e-14, so the
    dense case takes GMRES-IR (method 1), which needs the factors only as a
    preconditioner; the structured multipliers are checked with both."""
    n, nrhs = 256, 4
    A, _, B = (t.numpy() for t in W.shifted(1, n, nrhs, seed=4))
    A, B = A[0], B[0]
    X, info, G, F = g.solve_system(cu(A, torch.float32), cu(B), kind=kind, seed=2, prec=g.FP32, refine_steps=12,
                                   tol=1e-16, method=method)
    A32 = A.astype(np.float32).astype(np.float64)       # the matrix actually solved
    assert oracle.backward_error(A32, host(X), B) <= 1e-14
    assert info.bwd_err[0] > 1e-10                      # FP32 factors before refinement


# ---------------------------------------------------------------- adjoint

@pytest.mark.parametrize("kind", [0, 1, 2])
def test_adjoint_vs_oracle_gradient(g, kind):
    """dA, dB for loss sum(x^2) at n = 64 in FP64 against the oracle's
    gradient (lambda = A^{-T} gX by GEPP on A^T): relative error <= 1e-10."""
    n, nrhs = 64, 3
    A, _, B = (t.numpy() for t in W.shifted(1, n, nrhs, seed=7))
    A, B = A[0], B[0]
    X, info, G, F = g.solve_system(cu(A), cu(B), kind=kind, seed=3, refine_steps=5, tol=1e-17)
    x = host(X)
    gX = cu(2.0 * x)
    dA = torch.empty((n, n), dtype=torch.float64, device=DEV)
    dB = torch.empty((n, nrhs), dtype=torch.float64, device=DEV)
    g.adjoint(F, G, gX, X, dA, dB)
    dA_ref, dB_ref = oracle.adjoint(A, x, 2.0 * x)
    dA_g, dB_g = host(dA), host(dB)
    assert np.linalg.norm(dA_g - dA_ref) <= 1e-10 * np.linalg.norm(dA_ref)
    assert np.linalg.norm(dB_g - dB_ref) <= 1e-10 * np.linalg.norm(dB_ref)
    # entry by entry: dA = -Lambda X^T with the GPU's own Lambda = dB, so
    # |dA - dA_ref|_ij <= (|dB - dB_ref| |X|^T)_ij plus the rounding of the
    # two products (2 nrhs u (|Lambda| |X|^T)_ij)
    outer = np.abs(dB_ref) @ np.abs(x).T
    assert np.all(np.abs(dA_g - dA_ref) <= np.abs(dB_g - dB_ref) @ np.abs(x).T + 2 * nrhs * U * outer * 1.01)


def test_adjoint_independent_of_multiplier(g):
    n, nrhs = 96, 2
    A, _, B = (t.numpy() for t in W.shifted(1, n, nrhs, seed=8))
    A, B = A[0], B[0]
    grads = []
    for seed in (1, 2):
        X, _, G, F = g.solve_system(cu(A), cu(B), seed=seed, refine_steps=5, tol=1e-17)
        dA = torch.empty((n, n), dtype=torch.float64, device=DEV)
        g.adjoint(F, G, 2.0 * X, X, dA, None)
        grads.append(host(dA))
    assert np.linalg.norm(grads[0] - grads[1]) <= 1e-10 * np.linalg.norm(grads[0])


# ---------------------------------------------------------------- refinement as a CUDA graph

@pytest.mark.parametrize("method", [0, 1])
def test_refine_graph_matches_launch_by_launch(g, method):
    """genp_refine replayed from its cached CUDA graph solves as the
    launch-by-launch sequence does (the streaming triangular solves add
    their off-diagonal contributions with atomics, so two runs agree to
    rounding, not bit for bit), reports through the same status word, and a
    new right-hand side buffer records a new graph (keyed by the arguments).
    The graph's steps after convergence are IF-node bodies that it skips, so
    it launches fewer kernels: for the classic method exactly those of a
    launch-by-launch run stopped at the same step, plus one condition kernel
    per body (2 max_iter)."""
    lib = g._lib.load()
    n, nrhs = 300, 2
    A, _, B = (t.numpy() for t in W.lead_deficient(n, 32, 16, nrhs, seed=11))
    Ad, Bd = cu(A), cu(B)
    G = g.make_multiplier(g.GAUSSIAN, n, seed=4)
    C = torch.empty((n, n), dtype=torch.float64, device=DEV)
    g.precondition(G, Ad, C)
    F = g.factor(C)
    out = {}
    prev = lib.genp_refine_graphs(-1)
    X = torch.empty_like(Bd)
    X2 = torch.empty_like(Bd)
    try:
        # eager; the graph recorded, then replayed; a new X buffer (a new graph)
        for mode, Xb in ((0, X), (1, X), (1, X), (1, X2)):
            lib.genp_refine_graphs(mode)
            X = Xb
            g.solve(F, G, Bd, X)
            l0 = g.launch_count()
            g.refine(Ad, F, G, Bd, X, tol=1e-16, max_iter=6, method=method)
            info = g.info_fetch(F)
            out.setdefault(mode, []).append((host(X), info.bwd_err, info.refine_iters, g.launch_count() - l0))
    finally:
        lib.genp_refine_graphs(prev)
    x0, e0, i0, l_eager = out[0][0]
    assert oracle.backward_error(A, x0, B) <= 1e-14
    for x1, e1, i1, l_graph in out[1]:
        assert oracle.backward_error(A, x1, B) <= 1e-14
        assert np.abs(x1 - x0).max() <= 1e-12 * np.abs(x0).max()
        assert e1[-1] <= 1e-14 and abs(i1 - i0) <= 1
        assert l_graph > 0                    # the graph's kernels are counted when it runs
        if i1 < 5:
            assert l_graph < l_eager
    if method == 0:
        prev = lib.genp_refine_graphs(0)
        try:
            for _, _, i1, l_graph in out[1]:
                g.solve(F, G, Bd, X)
                l0 = g.launch_count()
                g.refine(Ad, F, G, Bd, X, tol=1e-16, max_iter=i1, method=0)
                assert l_graph == g.launch_count() - l0 + 2 * 6
        finally:
            lib.genp_refine_graphs(prev)

