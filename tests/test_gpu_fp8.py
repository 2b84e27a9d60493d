"""E4M3 operands with per-tile power-of-two scales (GENP_FP8_E4M3) vs the oracle.

* genp_quantize_e4m3: codes and tile scales bit for bit equal to the
  oracle's (integer work: the same rounding of the same exactly scaled
  values), FP32 and FP64 sources, both orientations, ragged edges, a zero
  tile, subnormal codes and exact ties;
* genp_gemm_e4m3: against the oracle's product of the same codes, exact in
  FP64 per k-tile.  The tensor cores accumulate a run of k-tiles with equal
  scale products in FP32 (fewer than K additions) and the promotion adds at
  most nkt FP32 multiply-adds, so
  |D - D_oracle| <= (K + nkt + 2) 2^-24 |alpha| sum_k |a_k b_k| + 2^-23 |beta C|;
  small integers are exact; runs of every length (scale patterns along K);
* the FP8 grid of a Gaussian multiplier bit for bit; C = A G on the e4m3
  tensor cores within the product bound;
* the factorization: |L U - C| <= (2^-3 + 2^-7) |L||U| elementwise (two
  e4m3 roundings of 2^-4 per Schur product, FP32 elsewhere) plus the
  subnormal codes' absolute error; bit-exact against the oracle's FP8
  blocked GENP on small-integer factors; GMRES-IR takes FP8 factors of a
  well-conditioned system of small growth to backward error <= 1e-14.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
U32 = 2.0 ** -24
FP64, FP32, FP8 = 0, 1, 3


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _s():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def quantize(lib, X, trans=False):
    """Codes (m x K) and scales of the logical operand X, or of X^T when trans."""
    src = X
    m, K = (src.shape[1], src.shape[0]) if trans else src.shape
    ldq = max(16, (K + 15) // 16 * 16)
    dst = torch.full((max(m, 1), ldq), 0xAB, dtype=torch.uint8, device=DEV)
    sc = torch.full((max(1, -(-m // 128)) * max(1, -(-K // 128)),), -1.0, dtype=torch.float32, device=DEV)
    prec = FP64 if src.dtype == torch.float64 else FP32
    st = lib.genp_quantize_e4m3(_p(src), src.stride(0), prec, m, K, int(trans), _p(dst), ldq, _p(sc), _s())
    assert st == 0, st
    torch.cuda.synchronize()
    assert lib.genp_device_check(1) == 0
    return dst, sc, ldq


def gemm(lib, Aq, sA, Bq, sB, m, n, K, alpha=1.0, beta=0.0, Cin=None, D=None):
    if D is None:
        D = torch.full((m, n), float("nan"), dtype=torch.float32, device=DEV)
    st = lib.genp_gemm_e4m3(m, n, K, alpha, _p(Aq), Aq.stride(0), _p(sA), _p(Bq), Bq.stride(0), _p(sB), beta,
                            _p(Cin), Cin.stride(0) if Cin is not None else 0, _p(D), D.stride(0), _s())
    assert st == 0, st
    torch.cuda.synchronize()
    assert lib.genp_device_check(1) == 0
    return D


def _operand(rng, m, K, spread=8.0):
    X = rng.standard_normal((m, K)) * np.exp2(rng.uniform(-spread, spread, (m, 1)))
    if m > 128 and K > 128:
        X[128:256, :128] = 0.0                          # a zero tile
    X[0, : min(K, 5)] = np.array([448.0, 464.0, 2.0 ** -10, 1.5 * 2.0 ** -9, -3.5 * 2.0 ** -9])[: min(K, 5)]
    return X


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("m,K", [(1, 1), (128, 128), (300, 257), (129, 1000), (5, 700)])
def test_quantize_bit_exact(genp_lib, dtype, trans, m, K):
    rng = np.random.default_rng(m * 7 + K)
    X = _operand(rng, m, K)
    if dtype == torch.float32:
        X = X.astype(np.float32).astype(np.float64)
    src = torch.as_tensor(X.T.copy() if trans else X).to(DEV, dtype)
    q, sc, ldq = quantize(genp_lib, src, trans)
    codes, scales = oracle.quantize_e4m3(X)
    assert np.array_equal(q.cpu().numpy()[:m, :K], codes)
    assert np.array_equal(sc.cpu().numpy().astype(np.float64), scales.reshape(-1))
    if ldq > K:                                          # columns past K are left alone
        assert np.all(q.cpu().numpy()[:m, K:] == 0xAB)


@pytest.mark.parametrize("m,n,K", [(128, 128, 128), (1, 1, 16), (200, 130, 72), (256, 384, 512), (515, 260, 1000),
                                   (130, 700, 1300)])
def test_gemm_matches_oracle(genp_lib, m, n, K):
    rng = np.random.default_rng(m + 3 * n + 5 * K)
    A = _operand(rng, m, K, 4.0)
    Bt = _operand(rng, n, K, 4.0)
    Aq, sA, _ = quantize(genp_lib, torch.as_tensor(A).to(DEV))
    Bq, sB, _ = quantize(genp_lib, torch.as_tensor(Bt).to(DEV))
    C = rng.standard_normal((m, n)).astype(np.float32)
    Cd = torch.as_tensor(C).to(DEV)
    D = gemm(genp_lib, Aq, sA, Bq, sB, m, n, K, alpha=-0.5, beta=2.0, Cin=Cd).cpu().double().numpy()
    codes_a, sa = oracle.quantize_e4m3(A)
    codes_b, sb = oracle.quantize_e4m3(Bt)
    ref = oracle.gemm_e4m3(codes_a, sa, codes_b, sb, alpha=-0.5, beta=2.0, C=C.astype(np.float64))
    absprod = np.abs(oracle.dequantize_e4m3(codes_a, sa)) @ np.abs(oracle.dequantize_e4m3(codes_b, sb)).T
    nkt = -(-K // 128)
    tol = (K + nkt + 2) * U32 * 0.5 * absprod + 2 * U32 * 2.0 * np.abs(C)
    assert np.all(np.abs(D - ref) <= tol)
    # typical error far below the worst case
    assert np.median(np.abs(D - ref) / np.maximum(0.5 * absprod, 1e-300)) < 16 * U32


@pytest.mark.parametrize("pattern", [[0, 0, 0, 0, 0], [0, 3, 0, 3, 0], [0, 0, -5, -5, -5], [2, 2, 2, 0, 7]])
def test_gemm_scale_runs(genp_lib, pattern):
    """Column blocks of A scaled by 2^p (p per k-tile): runs of equal tile
    scales of every length, each promoted with its own scale."""
    rng = np.random.default_rng(sum((p + 8) * 16 ** i for i, p in enumerate(pattern)))
    m, n = 256, 200
    K = 128 * len(pattern) - 40                       # ragged last k-tile
    A = rng.standard_normal((m, K))
    for kt, p in enumerate(pattern):
        A[:, 128 * kt:128 * (kt + 1)] *= 2.0 ** p
    Bt = rng.standard_normal((n, K))
    Aq, sA, _ = quantize(genp_lib, torch.as_tensor(A).to(DEV))
    Bq, sB, _ = quantize(genp_lib, torch.as_tensor(Bt).to(DEV))
    D = gemm(genp_lib, Aq, sA, Bq, sB, m, n, K).cpu().double().numpy()
    codes_a, sa = oracle.quantize_e4m3(A)
    codes_b, sb = oracle.quantize_e4m3(Bt)
    ref = oracle.gemm_e4m3(codes_a, sa, codes_b, sb)
    absprod = np.abs(oracle.dequantize_e4m3(codes_a, sa)) @ np.abs(oracle.dequantize_e4m3(codes_b, sb)).T
    assert np.all(np.abs(D - ref) <= (K + len(pattern) + 2) * U32 * absprod)


def test_gemm_small_integers_exact_and_inplace(genp_lib):
    rng = np.random.default_rng(1)
    m, n, K = 260, 300, 384
    A = rng.integers(-15, 16, (m, K)).astype(np.float64)
    B = rng.integers(-15, 16, (K, n)).astype(np.float64)
    Aq, sA, _ = quantize(genp_lib, torch.as_tensor(A).to(DEV))
    Bq, sB, _ = quantize(genp_lib, torch.as_tensor(B).to(DEV), trans=True)
    C0 = rng.integers(-1000, 1000, (m, n)).astype(np.float32)
    D = torch.as_tensor(C0).to(DEV)
    gemm(genp_lib, Aq, sA, Bq, sB, m, n, K, alpha=-1.0, beta=1.0, Cin=D, D=D)     # D <- D - A B
    assert np.array_equal(D.cpu().double().numpy(), C0.astype(np.float64) - A @ B)


@pytest.mark.parametrize("n", [64, 256, 1000])
def test_fp8_grid_multiplier_bit_exact(g, n):
    G = g.make_multiplier(g.GAUSSIAN, n, seed=9, value_grid=g.FP8_E4M3)
    Gd = torch.empty((n, n), dtype=torch.float64, device=DEV)
    g.multiplier_export(G, dense=Gd)
    M = oracle.multiplier(oracle.KIND_GAUSSIAN, n, seed=9, grid="fp32")
    assert np.array_equal(Gd.cpu().numpy(), oracle.fp8_grid(M["G"], 1.0 / np.sqrt(n)))


@pytest.fixture(scope="module")
def g(genp_lib):
    import paper_1212_4560_gb300 as genp
    assert genp_lib.genp_device_check(1) == 0
    return genp


@pytest.mark.parametrize("n", [128, 200, 520])
def test_precondition_e4m3(g, n):
    A, _, _ = W.lead_deficient(n, 16, 8, 1, seed=n)
    A = A.numpy()
    G = g.make_multiplier(g.GAUSSIAN, n, seed=2, value_grid=g.FP8_E4M3)
    Gd = torch.empty((n, n), dtype=torch.float64, device=DEV)
    g.multiplier_export(G, dense=Gd)
    Gm = Gd.cpu().numpy()
    C = torch.empty((n, n), dtype=torch.float32, device=DEV)
    g.precondition(G, torch.as_tensor(A).to(DEV), C, c_prec=g.FP8_E4M3)
    torch.cuda.synchronize()
    qa, sa = oracle.quantize_e4m3(A)
    qg, sg = oracle.quantize_e4m3(Gm.T.copy())
    assert np.array_equal(oracle.dequantize_e4m3(qg, sg), Gm.T)       # G on the grid: exact codes
    ref = oracle.gemm_e4m3(qa, sa, qg, sg)
    absprod = np.abs(oracle.dequantize_e4m3(qa, sa)) @ np.abs(Gm)
    nkt = -(-n // 128)
    assert np.all(np.abs(C.cpu().double().numpy() - ref) <= (128 + nkt + 2) * U32 * absprod)
    # and A G itself, within the e4m3 rounding of A
    assert np.all(np.abs(C.cpu().double().numpy() - A @ Gm) <= (2.0 ** -4 + 1e-5) * (np.abs(A) @ np.abs(Gm)) + 1e-6)


@pytest.mark.parametrize("n,nb", [(128, 0), (300, 0), (520, 128), (384, 64)])
def test_factor_e4m3_backward_error(g, n, nb):
    A, _, _ = W.lead_deficient(n, 16, 8, 1, seed=n + 1)
    C0 = oracle.precondition(A.numpy(), oracle.multiplier(0, n, seed=5)).astype(np.float32)
    C = torch.as_tensor(C0).to(DEV)
    F = g.factor(C, prec=g.FP8_E4M3, nb=nb)
    info = g.info_fetch(F)
    assert info.breakdown_step == -1
    assert g._lib.load().genp_device_check(1) == 0
    L, U = oracle.split_lu(C.cpu().double().numpy())
    E = np.abs(L @ U - C0.astype(np.float64))
    LU = np.abs(L) @ np.abs(U)
    # subnormal codes: absolute error <= 2^-10 s per operand, s <= amax / 224
    sub = 2 * 2.0 ** -10 / 224 * np.max(np.abs(L)) * np.max(np.abs(U)) * n
    assert np.all(E <= (2.0 ** -3 + 2.0 ** -7) * LU + sub)
    if n > 128:      # the Schur updates really ran at 8-bit precision
        assert np.max(E / np.maximum(LU, 1e-300)) > 1e-4


@pytest.mark.parametrize("n", [512, 2100])
def test_fp8_gmres_ir_reaches_fp64_accuracy(g, n):
    """Where the element growth is small, FP8 factors precondition GMRES-IR
    to eta <= 1e-14: plain GENP (identity multiplier) of a Gaussian matrix
    with a large diagonal shift, growth ~1.  (A Gaussian multiplier raises
    the growth of the same system to ~4e4, and 2^-4 times that is no
    preconditioner: the oracle's emulation of the FP8 factorization
    stagnates at eta ~0.1.)  n = 2100: 17 block steps with ragged tiles."""
    A, _, B = (t.numpy() for t in W.shifted(1, n, 2, seed=4))
    A, B = A[0], B[0]
    X, info, G, F = g.solve_system(torch.as_tensor(A).to(DEV), torch.as_tensor(B).to(DEV), kind=g.IDENTITY, seed=3,
                                   prec=g.FP8_E4M3, refine_steps=10, tol=1e-16, method=1)
    assert info.breakdown_step == -1
    assert info.growth < 4.0
    assert 1e-4 < info.bwd_err[0] < 0.1               # the unrefined FP8 solution is coarse
    eta = oracle.backward_error(A, X.cpu().numpy(), B)
    assert eta <= 1e-14
    assert g._lib.load().genp_device_check(1) == 0


def test_fp8_refinement_reports_its_error(g):
    """Pivot-free FP8 factors of the rank-deficient-leading-block workload:
    the status and backward errors the library reports match the oracle's
    measurement of the returned X (converged or not)."""
    n = 256
    A, _, B = (t.numpy() for t in W.lead_deficient(n, 32, 16, 1, seed=0))
    X, info, G, F = g.solve_system(torch.as_tensor(A).to(DEV), torch.as_tensor(B).to(DEV), kind=g.GAUSSIAN, seed=5,
                                   prec=g.FP8_E4M3, refine_steps=10, tol=1e-16, method=1)
    assert info.breakdown_step == -1
    eta = oracle.backward_error(A, X.cpu().numpy(), B)
    assert eta == pytest.approx(info.bwd_err[-1], rel=1e-6, abs=1e-15)
    assert g._lib.load().genp_device_check(1) == 0


@pytest.mark.parametrize("n,nb", [(300, 128), (256, 64)])
def test_factor_e4m3_small_integer_factors_bit_exact(g, n, nb):
    """C = L0 U0 with small integer factors (|L0| <= 2, |U0| <= 3, pivots
    +-1 or 2): every value the FP8 path forms is an integer exact in FP32,
    the block row and column are exact e4m3 values at every tile scale, so
    the GPU factors equal the oracle's FP8 blocked GENP, which equals L0 and
    U0, bit for bit."""
    rng = np.random.default_rng(8 + n)
    L0 = np.tril(rng.integers(-2, 3, (n, n)), -1) + np.eye(n)
    U0 = np.triu(rng.integers(-3, 4, (n, n)), 1) + np.diag(rng.choice([-1.0, 1.0, 2.0], n))
    C0 = L0 @ U0
    assert np.max(np.abs(C0)) < 2.0 ** 20
    LU_or, step = oracle.genp_fp8(C0, nb=nb)
    assert step == -1
    C = torch.as_tensor(C0).to(DEV, torch.float32)
    F = g.factor(C, prec=g.FP8_E4M3, nb=nb)
    assert g.info_fetch(F).breakdown_step == -1
    assert g._lib.load().genp_device_check(1) == 0
    assert np.array_equal(C.cpu().double().numpy(), LU_or)
