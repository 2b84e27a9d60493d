"""FP64-class products on the BF16 tensor cores (GENP_BF16_SLICED) vs the oracle.

The sliced product cuts each FP64 row of A and column of B, scaled by a power
of two 2^e > max|x|, into nd exact 7-bit digits and sums the digit products of
weight >= 2^-(7 nd + 7) on the tensor cores (K chunks of 512).  Error bounds
used below (per chunk, per term of the sum over k, against 2^{e_i + f_j}):
  operand truncation 2 * 2^-(7 nd + 1), dropped digit pairs (nd - 1) 2^-(7 nd + 2)
  and lower groups, FP32 rounding of the smallest group's accumulator,
so |D - A B|_ij <= 2^-(7 nd - 5) K max_k|a_ik| max_k|b_kj| (a factor of 8 to
spare over the sum of the terms above, which stay below 2^-(7 nd - 2)).  The
median relative error is also checked, at 2^-(7 nd - 5), which a wrong weight
or a lost digit group breaks by orders of magnitude.

Integer data whose rows need at most 7 nd bits slice exactly and sum exactly
(every group sum is an integer below 2^24), so C = L0 U0 with small-integer
factors must come back bit for bit, and a zero pivot made by the Schur update
must be exactly zero.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def cu(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dtype)


@pytest.fixture(scope="module")
def g(genp_lib):
    import paper_1212_4560_gb300 as genp
    assert genp_lib.genp_device_check(1) == 0
    return genp


@pytest.fixture
def digits(genp_lib, request):
    nd = request.param
    old = genp_lib.genp_sliced_digits(nd)
    assert old in (5, 6, 7)
    yield nd
    genp_lib.genp_sliced_digits(old)


def sliced(lib, A, B, alpha=1.0, beta=0.0, D=None, nd=0):
    m, K = A.shape
    n = B.shape[1]
    if D is None:
        D = torch.zeros((m, n), dtype=torch.float64, device=DEV)
    st = lib.genp_gemm_sliced(m, n, K, alpha, _p(A), A.stride(0), _p(B), B.stride(0), beta, _p(D), D.stride(0), nd,
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, st
    torch.cuda.synchronize()
    assert lib.genp_device_check(1) == 0
    return D


def bound(nd, A, B):
    K = A.shape[1]
    return 2.0 ** -(7 * nd - 5) * K * np.abs(A).max(1)[:, None] * np.abs(B).max(0)[None, :]


@pytest.mark.parametrize("nd", [3, 4, 5, 6, 7])
@pytest.mark.parametrize("m,n,K", [(1, 1, 1), (128, 64, 64), (200, 130, 1000), (77, 300, 513)])
def test_gemm_sliced_integers_exact(genp_lib, nd, m, n, K):
    rng = np.random.default_rng(m * 7 + n + K)
    A = rng.integers(-127, 128, (m, K)).astype(np.float64)
    B = rng.integers(-127, 128, (K, n)).astype(np.float64)
    D = sliced(genp_lib, cu(A), cu(B), nd=nd)
    assert np.array_equal(D.cpu().numpy(), oracle.matmul(A, B))


@pytest.mark.parametrize("nd", [3, 4, 5, 6, 7])
@pytest.mark.parametrize("m,n,K", [(128, 64, 512), (300, 260, 700), (129, 65, 1536)])
def test_gemm_sliced_gaussian(genp_lib, nd, m, n, K):
    rng = np.random.default_rng(nd * 1000 + K)
    A = rng.standard_normal((m, K)) * np.exp(rng.uniform(-3, 3, (m, 1)))    # rows of different scales
    B = rng.standard_normal((K, n)) * np.exp(rng.uniform(-3, 3, (1, n)))
    D = sliced(genp_lib, cu(A), cu(B), nd=nd).cpu().numpy()
    ref = oracle.matmul(A, B)
    err = np.abs(D - ref)
    assert np.all(err <= bound(nd, A, B))
    assert np.median(err / np.abs(ref)) <= 2.0 ** -(7 * nd - 5)


@pytest.mark.parametrize("nd", [3, 5, 7])
def test_gemm_sliced_schur_form_and_extremes(genp_lib, nd):
    """D <- D - A B in place, with every digit at its largest (entries
    0.999 give leading digits of 128 and the group sums reach 2^24 at K = 512)."""
    m, n, K = 140, 70, 1024
    A = np.full((m, K), 0.999)
    B = np.full((K, n), 0.999)
    D0 = np.random.default_rng(1).standard_normal((m, n))
    D = sliced(genp_lib, cu(A), cu(B), alpha=-1.0, beta=1.0, D=cu(D0), nd=nd).cpu().numpy()
    ref = D0 - oracle.matmul(A, B)
    assert np.all(np.abs(D - ref) <= bound(nd, A, B) + 2.0 ** -52 * np.abs(ref))


def test_gemm_sliced_rejects_bad_args(genp_lib):
    A = torch.zeros((4, 4), dtype=torch.float64, device=DEV)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert genp_lib.genp_gemm_sliced(4, 4, 4, 1.0, _p(A), 4, _p(A), 4, 0.0, _p(A), 4, 2, s) == -1   # 2 digits
    assert genp_lib.genp_gemm_sliced(4, 4, 4, 1.0, _p(A), 4, _p(A), 4, 0.0, _p(A), 4, 8, s) == -1   # 8 digits
    assert genp_lib.genp_gemm_sliced(4, 4, 4, 1.0, _p(A), 3, _p(A), 4, 0.0, _p(A), 4, 7, s) == -1   # lda < K
    assert genp_lib.genp_sliced_digits(4) == -1          # the factorization takes 5 to 7
    assert genp_lib.genp_sliced_digits(0) in (5, 6, 7)
    assert genp_lib.genp_sliced_precondition_digits(2) == -1
    assert genp_lib.genp_sliced_precondition_digits(8) == -1
    assert genp_lib.genp_sliced_precondition_digits(0) in (3, 4, 5, 6, 7)


@pytest.fixture
def pdigits(genp_lib, request):
    nd = request.param
    old = genp_lib.genp_sliced_precondition_digits(nd)
    assert old in (3, 4, 5, 6, 7)
    yield nd
    genp_lib.genp_sliced_precondition_digits(old)


@pytest.mark.parametrize("pdigits", [3, 4, 5, 7], indirect=True)
@pytest.mark.parametrize("n", [200, 1100])
def test_precondition_sliced(g, pdigits, n):
    digits = pdigits
    A, _, _ = W.lead_deficient(n, 32, 16, 1, seed=n)
    A = A.numpy()
    G = g.make_multiplier(g.GAUSSIAN, n, seed=3)
    Gd = torch.empty((n, n), dtype=torch.float64, device=DEV)
    g.multiplier_export(G, dense=Gd)
    Gm = Gd.cpu().numpy()
    C = torch.empty((n, n), dtype=torch.float64, device=DEV)
    g.precondition(G, cu(A), C, c_prec=g.BF16_SLICED)
    torch.cuda.synchronize()
    assert g._lib.load().genp_device_check(1) == 0
    ref = oracle.matmul(A, Gm)
    err = np.abs(C.cpu().numpy() - ref)
    assert np.all(err <= bound(digits, A, Gm))
    assert np.median(err / np.abs(ref)) <= 2.0 ** -(7 * digits - 5)


def _balanced(Lb, Ub):
    q = np.frexp(Lb.max(axis=0))[1].astype(float)
    r = (Lb * 2.0 ** -q[None, :]).max(axis=1)
    c = (Ub * 2.0 ** q[:, None]).max(axis=0)
    return r, c


def sliced_update_scale(L, U, nbo, nb):
    """S_ij = sum over the sliced products that update entry (i, j) of
    K max_k |l_ik| 2^-q_k max_k |u_kj| 2^q_k (k over the product's inner
    dimension, K its width).  A product L21 U12 is formed as
    (L21 D^-1)(D U12), D = diag(2^q_k) with q_k the least e such that
    max_i |l_ik| < 2^e over its L21 (frexp, 0 for a zero column), and its
    digit slices share one scale per row of L21 D^-1 and per column of
    D U12.  The products: each outer step's Schur update (K = nbo) of the
    trailing matrix, and, inside an outer step, the first inner step's
    update (K = nb) of the rest of the outer block column and of the block
    row beyond it."""
    n = L.shape[0]
    S = np.zeros((n, n))
    for k0 in range(0, n, nbo):
        e0 = min(k0 + nbo, n)
        for i0 in range(k0, e0, nb):
            j0 = min(i0 + nb, e0)
            if j0 >= e0 or j0 >= n:
                continue
            r, c = _balanced(np.abs(L[j0:, i0:j0]), np.abs(U[i0:j0, j0:]))
            # rows j0.. against columns j0..e0, and rows j0..e0 against columns e0..
            S[j0:, j0:e0] += (j0 - i0) * r[:, None] * c[None, :e0 - j0]
            S[j0:e0, e0:] += (j0 - i0) * r[:e0 - j0, None] * c[None, e0 - j0:]
        if e0 >= n:
            break
        r, c = _balanced(np.abs(L[e0:, k0:e0]), np.abs(U[k0:e0, e0:]))
        S[e0:, e0:] += (e0 - k0) * r[:, None] * c[None, :]
    return S


@pytest.mark.parametrize("digits", [5, 6, 7], indirect=True)
@pytest.mark.parametrize("n,nb", [(96, 0), (300, 0), (520, 128), (700, 64)])
def test_factor_sliced_backward_error(g, digits, n, nb):
    """|L U - C|_ij <= 2^-(7 nd - 6) S_ij + 3 n u_df |L||U|_ij + (n / nb + 2) u_df |C|_ij
    with u_df = 2^-46: each sliced update (outer Schur updates and the inner
    block updates) errs by the sliced product's 2^-(7 nd - 5) K against the
    row and column maxima of its balanced operands (S, see
    sliced_update_scale); the double-float diagonal blocks and block solves
    err as an LU in a 48-bit arithmetic (Higham, Thm. 9.3, u_df allowing two
    bits for the pair arithmetic), and the double-float trailing matrix
    rounds once per update."""
    A, _, _ = W.lead_deficient(n, 16, 8, 1, seed=n + 1)
    C0 = oracle.precondition(A.numpy(), oracle.multiplier(0, n, seed=5))
    C = cu(C0)
    F = g.factor(C, prec=g.BF16_SLICED, nb=nb)
    info = g.info_fetch(F)
    assert info.breakdown_step == -1
    assert g._lib.load().genp_device_check(1) == 0
    L, U = oracle.split_lu(C.cpu().numpy())
    nbo = max(512, 2 * (nb or 128))   # the library's outer step
    S = sliced_update_scale(L, U, nbo, nb or 128)
    u_df = 2.0 ** -46
    df = 3 * n * u_df * (np.abs(L) @ np.abs(U)) + (n / (nb or 128) + 2) * u_df * np.abs(C0)
    err = np.abs(L @ U - C0)
    assert np.all(err <= 2.0 ** -(7 * digits - 6) * S + df)
    # the bound is not slack by orders of magnitude: a lost digit group would pass it only at larger errors
    tail = S > 0
    if tail.any():
        assert np.median(err[tail] / S[tail]) <= 2.0 ** -(7 * digits)


@pytest.mark.parametrize("digits", [5, 7], indirect=True)
@pytest.mark.parametrize("n", [128, 257, 400])
def test_factor_sliced_integer_exact(g, digits, n):
    rng = np.random.default_rng(n)
    L0 = np.tril(rng.integers(-2, 3, (n, n)), -1) + np.eye(n, dtype=np.int64)
    U0 = np.triu(rng.integers(-2, 3, (n, n)), 1) + np.diag(rng.choice([-1, 1], n))
    C0 = (L0 @ U0).astype(np.float64)
    C = cu(C0)
    F = g.factor(C, prec=g.BF16_SLICED, nb=64)
    assert g.info_fetch(F).breakdown_step == -1
    L, U = oracle.split_lu(C.cpu().numpy())
    assert np.array_equal(L, L0.astype(float))
    assert np.array_equal(U, U0.astype(float))


def test_factor_sliced_breakdown_after_schur_update(g):
    """u_kk = 0 exactly at k = 130 (inside the third panel of 64): the zero is
    produced by the sliced Schur updates, which must be exact on integers."""
    n, k = 256, 130
    rng = np.random.default_rng(5)
    L0 = np.tril(rng.integers(-2, 3, (n, n)), -1) + np.eye(n, dtype=np.int64)
    d = rng.choice([-1, 1], n)
    d[k] = 0
    U0 = np.triu(rng.integers(-2, 3, (n, n)), 1) + np.diag(d)
    C = cu((L0 @ U0).astype(np.float64))
    F = g.factor(C, prec=g.BF16_SLICED, nb=64)
    info = g.info_fetch(F)
    assert info.breakdown_step == k
    assert info.status == -2      # GENP_ERR_BREAKDOWN


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_sliced_with_fp64_refinement(g, kind):
    A, _, B = (t.numpy() for t in W.lead_deficient(256, 32, 16, 1, seed=0))
    X, info, G, F = g.solve_system(cu(A), cu(B), kind=kind, seed=5, prec=g.BF16_SLICED, refine_steps=10, tol=1e-16)
    eta = oracle.backward_error(A, X.cpu().numpy(), B)
    assert eta <= 1e-14
    assert info.breakdown_step == -1
    assert g._lib.load().genp_device_check(1) == 0


@pytest.mark.parametrize("digits", [7], indirect=True)
@pytest.mark.parametrize("kappa", [1e2, 1e6])
def test_sliced_ill_conditioned(g, digits, kappa):
    n = 1024
    A, Xs, B = (t.numpy() for t in W.svd_kappa(n, kappa, 1, seed=1))
    X, info, G, F = g.solve_system(cu(A), cu(B), kind=g.GAUSSIAN, seed=2, prec=g.BF16_SLICED, refine_steps=15,
                                   tol=1e-16)
    x = X.cpu().numpy()
    assert oracle.backward_error(A, x, B) <= 1e-14
    assert np.abs(x - Xs).max() / np.abs(Xs).max() <= 1e-14 * kappa * 10


def test_sliced_adjoint(g):
    n, nrhs = 160, 2
    A, _, B = (t.numpy() for t in W.shifted(1, n, nrhs, seed=4))
    A, B = A[0], B[0]
    X, info, G, F = g.solve_system(cu(A), cu(B), kind=g.GAUSSIAN, seed=1, prec=g.BF16_SLICED, refine_steps=10,
                                   tol=1e-16)
    dA = torch.empty((n, n), dtype=torch.float64, device=DEV)
    dB = torch.empty((n, nrhs), dtype=torch.float64, device=DEV)
    g.adjoint(F, G, X, X, dA, dB)
    x = X.cpu().numpy()
    dA_ref, dB_ref = oracle.adjoint(A, x, x)
    # the adjoint reuses the sliced factors without refinement: its error is
    # the factorization's (2^-46 against the operand scales, times the growth
    # and the conditioning), far below the 1e-6 of the gradient check
    assert np.linalg.norm(dB.cpu().numpy() - dB_ref) <= 1e-6 * np.linalg.norm(dB_ref)
    assert np.linalg.norm(dA.cpu().numpy() - dA_ref) <= 1e-6 * np.linalg.norm(dA_ref)


@pytest.mark.parametrize("digits", [5, 6, 7], indirect=True)
@pytest.mark.parametrize("kappa", [1e2, 1e6])
def test_sliced_gmres_ir(g, digits, kappa):
    """GMRES-IR (genp_refine method 1) needs the factors only as a
    preconditioner: 5 and 6 digits, where classic refinement stalls on the
    kappa = 1e6 system, still reach eta <= 1e-14 in a few outer steps."""
    n = 1024
    A, Xs, B = (t.numpy() for t in W.svd_kappa(n, kappa, 1, seed=1))
    X, info, G, F = g.solve_system(cu(A), cu(B), kind=g.GAUSSIAN, seed=2, prec=g.BF16_SLICED, refine_steps=6,
                                   tol=1e-16, method=1)
    x = X.cpu().numpy()
    assert oracle.backward_error(A, x, B) <= 1e-14
    assert np.abs(x - Xs).max() / np.abs(Xs).max() <= 1e-14 * kappa * 10
    assert info.refine_iters <= 4
    assert g._lib.load().genp_device_check(1) == 0


@pytest.mark.parametrize("pdigits", [4, 5], indirect=True)
@pytest.mark.parametrize("digits", [7], indirect=True)
def test_sliced_gmres_ir_short_precondition(g, digits, pdigits):
    """A G from 4 or 5 digits (genp_sliced_precondition_digits) and 7-digit
    factors: GMRES-IR, with the FP64 residual on A and the FP64 update with
    G, still takes the kappa = 1e6 system to eta <= 1e-14."""
    n = 1024
    A, Xs, B = (t.numpy() for t in W.svd_kappa(n, 1e6, 1, seed=3))
    X, info, G, F = g.solve_system(cu(A), cu(B), kind=g.GAUSSIAN, seed=4, prec=g.BF16_SLICED, refine_steps=6,
                                   tol=1e-16, method=1)
    x = X.cpu().numpy()
    assert oracle.backward_error(A, x, B) <= 1e-14
    assert np.abs(x - Xs).max() / np.abs(Xs).max() <= 1e-14 * 1e6 * 10
    assert info.refine_iters <= 4
    assert g._lib.load().genp_device_check(1) == 0


# ------------------------------------------------ G on the sliced product's grid

class _mult_digits:
    """genp_sliced_multiplier_digits set for the multipliers made inside."""

    def __init__(self, g, d):
        self.lib, self.d = g._lib.load(), d

    def __enter__(self):
        self.prev = self.lib.genp_sliced_multiplier_digits(self.d)
        assert self.prev in (1, 2)

    def __exit__(self, *exc):
        self.lib.genp_sliced_multiplier_digits(self.prev)


def test_multiplier_digits_setting(g):
    """genp_sliced_multiplier_digits: 1 by default, 1 or 2 accepted, anything
    else refused with -1 and the setting kept."""
    lib = g._lib.load()
    assert lib.genp_sliced_multiplier_digits(0) == 1
    assert lib.genp_sliced_multiplier_digits(3) == -1
    assert lib.genp_sliced_multiplier_digits(-2) == -1
    assert lib.genp_sliced_multiplier_digits(2) == 1
    assert lib.genp_sliced_multiplier_digits(1) == 2
    assert lib.genp_sliced_multiplier_digits(0) == 1


@pytest.mark.parametrize("digits", [1, 2])
@pytest.mark.parametrize("n", [64, 257, 1024])
def test_sliced_grid_multiplier_bit_exact(g, n, digits):
    """value_grid GENP_BF16_SLICED: the single precision draw rounded to
    multiples of 2^(E - 7 digits + 1) for the dense Gaussian (2^(E - 13) for
    the circulant), bit for bit the oracle's; a redraw keeps the grid."""
    s = 1.0 / np.sqrt(n)
    with _mult_digits(g, digits):
        G = g.make_multiplier(g.GAUSSIAN, n, seed=n, value_grid=g.BF16_SLICED)
    D = torch.empty((n, n), dtype=torch.float64, device=DEV)
    g.multiplier_export(G, dense=D)
    ref = oracle.sliced_grid(oracle.multiplier(0, n, seed=n, grid="fp32")["G"], s, digits=digits)
    assert np.array_equal(D.cpu().numpy(), ref)
    with _mult_digits(g, 3 - digits):
        g.redraw_multiplier(G, seed=n + 1)
    g.multiplier_export(G, dense=D)
    ref = oracle.sliced_grid(oracle.multiplier(0, n, seed=n + 1, grid="fp32")["G"], s, digits=digits)
    assert np.array_equal(D.cpu().numpy(), ref)
    Gc = g.make_multiplier(g.CIRCULANT, n, seed=n, value_grid=g.BF16_SLICED)
    col = torch.empty(n, dtype=torch.float64, device=DEV)
    g.multiplier_export(Gc, first_col=col)
    ref_c = oracle.sliced_grid(oracle.multiplier(1, n, seed=n, grid="fp32")["g"], 1.0)
    assert np.array_equal(col.cpu().numpy(), ref_c)


@pytest.mark.parametrize("mdigits", [1, 2])
@pytest.mark.parametrize("pdigits", [5, 7], indirect=True)
@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("n", [300, 1100])
def test_precondition_two_digit_multiplier(g, pdigits, side, n, mdigits):
    """With G on the sliced grid, A G (and G A) take G in its one or two
    digits (7 or 13 digit products for 7 digits of A instead of 28): the
    same error bound as the symmetric product, against the oracle's FP64
    product of the same G."""
    digits = pdigits
    A, _, _ = W.lead_deficient(n, 32, 16, 1, seed=n + 7)
    A = A.numpy()
    with _mult_digits(g, mdigits):
        G = g.make_multiplier(g.GAUSSIAN, n, seed=9, value_grid=g.BF16_SLICED, side=side)
    Gd = torch.empty((n, n), dtype=torch.float64, device=DEV)
    g.multiplier_export(G, dense=Gd)
    Gm = Gd.cpu().numpy()
    C = torch.empty((n, n), dtype=torch.float64, device=DEV)
    g.precondition(G, cu(A), C, c_prec=g.BF16_SLICED)
    torch.cuda.synchronize()
    assert g._lib.load().genp_device_check(1) == 0
    if side == 0:
        ref, bnd = oracle.matmul(A, Gm), bound(digits, A, Gm)
    else:
        ref, bnd = oracle.matmul(Gm, A), bound(digits, Gm, A)
    err = np.abs(C.cpu().numpy() - ref)
    assert np.all(err <= bnd)
    assert np.median(err / np.abs(ref)) <= 2.0 ** -(7 * digits - 5)


@pytest.mark.parametrize("kappa", [1e2, 1e6])
def test_sliced_grid_gmres_ir_end_to_end(g, kappa):
    """The benchmark's arithmetic at n = 1024: G on the sliced grid, 7-digit
    factors, GMRES-IR to eta <= 1e-14 (oracle backward error) and the forward
    error within 1e-14 kappa_2 (x10 for the inf-norm)."""
    n = 1024
    A, Xs, B = (t.numpy() for t in W.svd_kappa(n, kappa, 1, seed=5))
    Ad, Bd = cu(A), cu(B)
    G = g.make_multiplier(g.GAUSSIAN, n, seed=6, value_grid=g.BF16_SLICED)
    C = torch.empty((n, n), dtype=torch.float64, device=DEV)
    g.precondition(G, Ad, C, c_prec=g.BF16_SLICED)
    F = g.factor(C, prec=g.BF16_SLICED)
    X = torch.empty_like(Bd)
    g.solve(F, G, Bd, X)
    g.refine(Ad, F, G, Bd, X, tol=1e-16, max_iter=6, method=1)
    info = g.info_fetch(F)
    x = X.cpu().numpy()
    assert info.breakdown_step == -1
    assert oracle.backward_error(A, x, B) <= 1e-14
    assert np.abs(x - Xs).max() / np.abs(Xs).max() <= 1e-14 * kappa * 10
    assert info.refine_iters <= 4


def test_profile_classes_report_the_launches(g):
    """genp_profile_class: with the profile on, a sliced solve records its
    tensor-core launches (class 0: work = the FP64-class products' 2 m n K,
    at least A G's 2 n^3 and the Schur updates' 2 (n - 256)^3 / 3 when
    n > 256), triangular solves (class 1: n^2 / 2 x 8 bytes for each launch
    that ran, fewer when refinement launches were skipped) and
    matrix-vector products (class 2); class 6 does not exist."""
    import ctypes
    lib = g._lib.load()
    n = 700
    A, _, B = (t.numpy() for t in W.svd_kappa(n, 1e4, 1, seed=2))
    prev = lib.genp_refine_graphs(0)      # launch by launch, so the profile sees the refinement
    lib.genp_profile_enable(1)
    try:
        X, info, G, F = g.solve_system(cu(A), cu(B), kind=g.GAUSSIAN, seed=3, prec=g.BF16_SLICED, refine_steps=4,
                                       tol=1e-16, method=1)
        torch.cuda.synchronize()
        got = {}
        for cls in range(6):
            ms, w, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
            assert lib.genp_profile_class(cls, ctypes.byref(ms), ctypes.byref(w), ctypes.byref(c)) == 0
            got[cls] = (ms.value, w.value, c.value)
        ms, w, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        assert lib.genp_profile_class(6, ctypes.byref(ms), ctypes.byref(w), ctypes.byref(c)) == -1
    finally:
        lib.genp_profile_enable(0)
        lib.genp_refine_graphs(prev)
    t_ms, t_work, t_n = got[0]
    assert t_n > 0 and t_ms > 0
    assert t_work >= 2.0 * n**3 + 2.0 * (n - 256) ** 3 / 3
    assert t_work <= 2.0 * 768**3 + 2.0 * 768**3        # padded K at most
    s_ms, s_work, s_n = got[1]
    assert s_n >= 2 and s_ms > 0
    assert 0 < s_work <= s_n * 0.5 * n * n * 8 + 1
    assert got[2][2] > 0 and got[2][1] > 0
    assert oracle.backward_error(A, X.cpu().numpy(), B) <= 1e-14
