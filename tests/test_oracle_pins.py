"""Pins of the CPU oracle to things other than itself (runs without a GPU).

Each test fixes one function of ``oracle/`` against an independent
implementation, a closed form, an exact (rational) computation, an
invariant or a theorem of the paper, chosen so that a dropped term, a wrong
sign or index, or a transposed operand fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.stats as st
from fractions import Fraction

import oracle
import workloads as W

U64 = 2**64 - 1


# ---------------------------------------------------------------- generator

@pytest.mark.parametrize("ctr,key", [
    ([0, 0, 0, 0], [0, 0]),
    ([1, 2, 3, 4], [5, 6]),
    ([U64, U64, U64, U64], [U64, U64]),
    ([0x243F6A8885A308D3, 0x13198A2E03707344, 0xA4093822299F31D0, 0x082EFA98EC4E6C89],
     [0x452821E638D01377, 0xBE5466CF34E90C6C]),
    ([12345, 0, 0x10, 0], [2024, 7]),
])
def test_philox_matches_numpy(ctr, key):
    """Philox4x64-10 against NumPy's independent implementation.  NumPy
    increments its 256-bit counter before each block, so it is started one
    below the counter we want."""
    c = int(ctr[0]) | (int(ctr[1]) << 64) | (int(ctr[2]) << 128) | (int(ctr[3]) << 192)
    c = (c - 1) % (2**256)
    cw = np.array([(c >> (64 * i)) & U64 for i in range(4)], dtype=np.uint64)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=cw)
    ref = bg.random_raw(4)
    got = oracle.philox4x64_10(ctr, key)
    assert np.array_equal(got, ref)


def test_u53_exact():
    assert oracle.lib().or_u53(0) == 0.0
    assert oracle.lib().or_u53(U64) == 1.0 - 2.0**-53
    assert oracle.lib().or_u53(1 << 11) == 2.0**-53


def test_own_log_accuracy():
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.uniform(2**-60, 1.0, 20000), 2.0 ** -rng.uniform(0, 100, 2000),
                         [0.5, 0.25, 1.0 - 2**-53, 2**-104, 0.7071067811865476, 0.7071067811865475]])
    for x in xs:
        got = oracle.log(float(x))
        ref = math.log(float(x))
        if ref == 0.0:
            assert got == 0.0
        else:
            assert abs(got - ref) <= 2.5 * abs(ref) * 2**-52, (x, got, ref)
    # exact powers of two: ln(2^-k) = -k ln 2 (f = 0 exactly)
    for k in range(1, 60):
        assert oracle.log(2.0**-k) == -k * 0.6931471805599453


def test_gaussian_distribution():
    """Dense multiplier entries are N(0, scale^2): moments and a KS test on
    250k samples; scale = 1/sqrt(n) (variance 1/n)."""
    n = 500
    G = oracle.multiplier(0, n, seed=11)["G"]
    z = G.ravel() * math.sqrt(n)
    assert abs(z.mean()) < 0.01
    assert abs(z.std() - 1.0) < 0.01
    assert abs(st.skew(z)) < 0.02
    assert abs(st.kurtosis(z)) < 0.05
    assert st.kstest(z, "norm").pvalue > 1e-3
    # entries of a different seed / stream differ
    G2 = oracle.multiplier(0, n, seed=11, stream=1)["G"]
    assert not np.any(G2 == G)


def test_own_log_f32_accuracy():
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.uniform(2**-40, 1.0, 20000).astype(np.float32), [0.5, 0.25, 1 - 2**-24]])
    for x in xs:
        x = float(np.float32(x))
        got, ref = oracle.log_f32(x), math.log(x)
        assert abs(got - ref) <= 3 * abs(ref) * 2**-23 + 1e-45, (x, got, ref)
    for k in range(1, 40):
        assert oracle.log_f32(2.0**-k) == float(np.float32(-k * np.float32(0.693147182)))


def test_gaussian_f32_distribution():
    """Single-precision draws: moments and KS on 250k samples, values on the
    FP32 grid, scale rounded to float."""
    n = 500
    G = oracle.multiplier(0, n, seed=13, grid="fp32")["G"]
    assert np.array_equal(G.astype(np.float32).astype(np.float64), G)
    z = G.ravel() / float(np.float32(1 / math.sqrt(n)))
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    assert st.kstest(z, "norm").pvalue > 1e-3
    # one entry recomputed with numpy float32 arithmetic from the raw words
    w = oracle.philox4x64_10([0, 0, 0x14, 0], [13, 0])
    for p in range(2):
        u1 = np.float32(int(w[2 * p]) >> 40) * np.float32(2.0**-24)
        u2 = np.float32(int(w[2 * p + 1]) >> 40) * np.float32(2.0**-24)
        v1, v2 = np.float32(2) * u1 - np.float32(1), np.float32(2) * u2 - np.float32(1)
        s = v1 * v1 + v2 * v2
        if 0 < s < 1:
            ref = float(v1) * math.sqrt(-2 * math.log(float(s)) / float(s))
            got = oracle.gauss_f32(13, 0, 0x14, 0)
            assert abs(got - ref) <= 8 * abs(ref) * 2**-23
            break


def test_polar_method_by_hand():
    """Recompute one entry's polar step from the raw Philox words with
    math.log / math.sqrt; equal to within 2 ulp of the result."""
    seed, stream, tag, idx = 99, 3, 0x10, 17
    for blk in range(32):
        w = oracle.philox4x64_10([idx, blk, tag, 0], [seed, stream])
        for p in range(2):
            v1 = 2.0 * ((int(w[2 * p]) >> 11) * 2.0**-53) - 1.0
            v2 = 2.0 * ((int(w[2 * p + 1]) >> 11) * 2.0**-53) - 1.0
            s = v1 * v1 + v2 * v2
            if 0.0 < s < 1.0:
                ref = v1 * math.sqrt(-2.0 * math.log(s) / s)
                got = oracle.gauss(seed, stream, tag, idx)
                assert abs(got - ref) <= 4 * abs(ref) * 2**-52
                return
    pytest.fail("no accepted pair")


def test_circulant_structure():
    n = 37
    M = oracle.multiplier(1, n, seed=5)
    g, G = M["g"], M["G"]
    assert np.array_equal(G[:, 0], g)                    # first column is g
    for i in range(n):
        for j in range(n):
            assert G[i, j] == G[(i + 1) % n, (j + 1) % n]  # wrap-around Toeplitz
    assert abs(g.std() - 1.0) < 0.5


def test_sparse_structure_and_uniformity():
    n = 64
    M = oracle.multiplier(2, n, seed=3)
    rows, signs, G = M["rows"], M["signs"], M["G"]
    for t in range(4):
        assert sorted(rows[t].tolist()) == list(range(n))   # each P_t is a permutation
    assert set(np.unique(signs).tolist()) <= {-1, 1}
    # column j holds exactly the signed entries it was given (with coincidences added)
    ref = np.zeros((n, n))
    for t in range(4):
        for j in range(n):
            ref[rows[t, j], j] += signs[t, j]
    assert np.array_equal(ref, G)
    assert np.array_equal(np.abs(G).sum(0) <= 4, np.ones(n, bool))
    # every row receives 4 entries counting multiplicity
    cnt = np.zeros(n, int)
    for t in range(4):
        np.add.at(cnt, rows[t], 1)
    assert np.all(cnt == 4)
    # Fisher-Yates over many seeds: all 24 permutations of 4 equally likely
    counts = {}
    for s in range(2400):
        r = tuple(oracle.multiplier(2, 4, seed=1000 + s, nnz=1)["rows"][0].tolist())
        counts[r] = counts.get(r, 0) + 1
    assert len(counts) == 24
    assert st.chisquare(list(counts.values())).pvalue > 1e-3


def test_thm41_tail_frequency():
    """Thm. 4.1 (MH form): Prob{||(MH)^+|| >= 2.35 x sqrt(r) ||M^+|| / sigma} <= 1/x
    for Gaussian H with entry std sigma.  Checked as a frequency over seeds."""
    n, x, trials = 24, 4.0, 200
    rng = np.random.default_rng(1)
    Mmat = rng.standard_normal((n, n))
    Mp = np.linalg.norm(np.linalg.pinv(Mmat), 2)
    sigma = 1.0 / math.sqrt(n)
    bad = 0
    for s in range(trials):
        H = oracle.multiplier(0, n, seed=s)["G"]
        P = Mmat @ H
        if np.linalg.norm(np.linalg.pinv(P), 2) >= 2.35 * x * math.sqrt(n) * Mp / sigma:
            bad += 1
    assert st.binomtest(bad, trials, 1.0 / x, alternative="greater").pvalue > 1e-3
    # Cor. 4.1 (ii) for leading k x k blocks of M H, in terms of the first k rows of M:
    # again a probability bound, checked as a frequency over seeds.
    Hs = [oracle.multiplier(0, n, seed=500 + s)["G"] for s in range(trials)]
    for k in (1, 3, 12, n):
        bound = 2.35 * x * math.sqrt(k) * np.linalg.norm(np.linalg.pinv(Mmat[:k]), 2) / sigma
        bad = sum(np.linalg.norm(np.linalg.pinv((Mmat @ H)[:k, :k]), 2) >= bound for H in Hs)
        assert st.binomtest(int(bad), trials, 1.0 / x, alternative="greater").pvalue > 1e-3


# ---------------------------------------------------------------- products

def test_matmul_integer_exact():
    rng = np.random.default_rng(2)
    A = rng.integers(-8, 9, (33, 45))
    B = rng.integers(-8, 9, (45, 29))
    C = oracle.matmul(A.astype(float), B.astype(float))
    assert np.array_equal(C, (A @ B).astype(float))       # int64 product is exact


def test_matmul_not_transposed():
    A = np.array([[1.0, 2.0], [0.0, 0.0]])
    B = np.array([[0.0, 1.0], [0.0, 0.0]])
    assert np.array_equal(oracle.matmul(A, B), np.array([[0.0, 1.0], [0.0, 0.0]]))


def test_circulant_products_vs_fft():
    """C = A G and G y for circulant G, against the convolution theorem."""
    n = 48
    rng = np.random.default_rng(3)
    M = oracle.multiplier(1, n, seed=9)
    g = M["g"]
    A = rng.standard_normal((5, n))
    C = oracle.precondition(A, M)
    # c_j = sum_i a_i g_{i-j} is a circular cross-correlation: fft(c) = fft(a) conj(fft(g))
    ref = np.real(np.fft.ifft(np.fft.fft(A, axis=1) * np.conj(np.fft.fft(g))[None, :], axis=1))
    assert np.allclose(C, ref, rtol=0, atol=1e-12 * np.abs(A).sum() * np.abs(g).max())
    Y = rng.standard_normal((n, 3))
    X = oracle.apply_multiplier(M, Y)
    refx = np.real(np.fft.ifft(np.fft.fft(g)[:, None] * np.fft.fft(Y, axis=0), axis=0))
    assert np.allclose(X, refx, atol=1e-12 * 100)
    XT = oracle.apply_multiplier(M, Y, trans=True)
    assert np.allclose(XT, M["G"].T @ Y, atol=1e-12)


def test_sparse_products_vs_scipy():
    n = 40
    rng = np.random.default_rng(4)
    M = oracle.multiplier(2, n, seed=21)
    cols = np.tile(np.arange(n), 4)
    S = sp.coo_matrix((M["signs"].ravel().astype(float), (M["rows"].ravel(), cols)), shape=(n, n)).tocsr()
    A = rng.standard_normal((7, n))
    assert np.allclose(oracle.precondition(A, M), (S.T @ A.T).T, atol=1e-13)
    Y = rng.standard_normal((n, 2))
    assert np.allclose(oracle.apply_multiplier(M, Y), S @ Y, atol=1e-13)
    assert np.allclose(oracle.apply_multiplier(M, Y, trans=True), S.T @ Y, atol=1e-13)
    # row-subset product equals the same rows of the full product
    C = oracle.precondition(A, M)
    assert np.array_equal(oracle.precondition(A, M, rows=[2, 5]), C[[2, 5]])


# ---------------------------------------------------------------- GENP / GEPP

def _integer_LU(n, rng):
    L0 = np.tril(rng.integers(-3, 4, (n, n)), -1) + np.eye(n, dtype=np.int64)
    U0 = np.triu(rng.integers(-3, 4, (n, n)), 1) + np.diag(rng.choice([-1, 1], n))
    return L0, U0


@pytest.mark.parametrize("n", [1, 2, 5, 16, 40])
def test_genp_recovers_integer_factors(n):
    """C = L0 U0 with unit-lower integer L0 and integer U0 with +-1 diagonal:
    every intermediate is a small integer, so GENP must return L0, U0 exactly
    (the pivot-free LU is unique when the leading minors are nonzero)."""
    rng = np.random.default_rng(n)
    L0, U0 = _integer_LU(n, rng)
    C = (L0 @ U0).astype(float)
    assert np.abs(C).max() < 2**40
    LU, k = oracle.genp(C)
    assert k == -1
    L, U = oracle.split_lu(LU)
    assert np.array_equal(L, L0.astype(float))
    assert np.array_equal(U, U0.astype(float))


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_pivots_vs_leibniz(n):
    """u_kk = det(C_k) / det(C_{k-1}) and prod u_kk = det(C) = det(A) det(G),
    all determinants by exact Leibniz expansion in rationals.  The first
    seed from 100 + n whose A and G are nonsingular and whose C has no
    singular leading minor is taken, so that every order runs."""
    for seed in range(100 + n, 100 + n + 50):
        rng = np.random.default_rng(seed)
        A = rng.integers(-4, 5, (n, n)).astype(float)
        A[0, 0] = 0.0                              # plain GENP on A would break down
        G = rng.integers(-4, 5, (n, n)).astype(float)
        C = oracle.matmul(A, G)                    # exact: small integers
        assert np.array_equal(C, (A.astype(np.int64) @ G.astype(np.int64)).astype(float))
        dA, dG = oracle.det_leibniz(A), oracle.det_leibniz(G)
        minors = [Fraction(1)] + [oracle.det_leibniz(C[:k, :k]) for k in range(1, n + 1)]
        if dA != 0 and dG != 0 and all(m != 0 for m in minors):
            break
    else:
        raise AssertionError("no nonsingular draw in 50 seeds")
    LU, k = oracle.genp(C)
    assert k == -1
    piv = np.diag(LU)
    for j in range(n):
        exact = minors[j + 1] / minors[j]
        assert abs(piv[j] - float(exact)) <= 1e-12 * abs(float(exact))
    prod = Fraction(1)
    for p in piv:
        prod *= Fraction(float(p))
    assert abs(float(prod) - float(dA * dG)) <= 1e-11 * abs(float(dA * dG))
    assert minors[n] == dA * dG


def test_thm22_pivot_bounds():
    """Thm. 2.2: every GENP pivot satisfies |u_kk| <= N + N_- N^2 and
    1/|u_kk| <= N_-, with N = ||C|| and N_- = max_j ||(C_j^(j))^{-1}||."""
    for seed in range(5):
        A, _, _ = W.lead_deficient(64, 8, 4, 1, seed)
        M = oracle.multiplier(0, 64, seed=seed)
        C = oracle.precondition(A.numpy(), M)
        N = np.linalg.norm(C, 2)
        Nm = max(np.linalg.norm(np.linalg.inv(C[:j, :j]), 2) for j in range(1, 65))
        LU, k = oracle.genp(C)
        assert k == -1
        piv = np.abs(np.diag(LU))
        assert piv.max() <= (N + Nm * N * N) * (1 + 1e-10)
        assert (1.0 / piv).max() <= Nm * (1 + 1e-8)


def test_genp_lu_reproduces_input():
    A, _, _ = W.lead_deficient(128, 16, 8, 1, 0)
    C = oracle.precondition(A.numpy(), oracle.multiplier(0, 128, seed=1))
    LU, k = oracle.genp(C)
    L, U = oracle.split_lu(LU)
    assert np.linalg.norm(L @ U - C) / np.linalg.norm(C) < 128 * 2**-52 * 100


def test_genp_breaks_down_on_2x2_and_multiplier_repairs():
    A = np.array([[0.0, 1.0], [1.0, 0.0]])
    LU, k = oracle.genp(A)
    assert k == 0
    b = np.array([[2.0], [3.0]])
    M = oracle.multiplier(0, 2, seed=4)
    r = oracle.solve(A, b, M, refine_steps=2, tol=1e-16)
    assert r["step"] == -1
    assert np.allclose(r["x"], [[3.0], [2.0]], rtol=0, atol=1e-14)


def test_gepp_equals_genp_on_column_dominant():
    """Column diagonally dominant => GEPP swaps nothing and, with the same
    update order, equals GENP bit for bit."""
    rng = np.random.default_rng(7)
    n = 50
    A = rng.standard_normal((n, n))
    A[np.diag_indices(n)] = np.abs(A).sum(0) + 1.0
    LU1, k1 = oracle.genp(A)
    LU2, piv, k2 = oracle.gepp(A)
    assert k1 == k2 == -1
    assert np.array_equal(piv, np.arange(n))
    assert np.array_equal(LU1, LU2)


def test_gepp_solve_vs_lapack():
    rng = np.random.default_rng(8)
    A = rng.standard_normal((60, 60))
    B = rng.standard_normal((60, 3))
    X = oracle.gepp_solve(A, B)
    assert np.allclose(X, sla.solve(A, B), rtol=1e-11, atol=1e-12)
    XT = oracle.gepp_solve_T(A, B)
    assert np.allclose(XT, sla.solve(A.T, B), rtol=1e-11, atol=1e-12)
    # the pivot choice is the first max (LAPACK idamax): compare with getrf
    lu, piv = sla.lu_factor(A)
    _, mypiv, _ = oracle.gepp(A)
    assert np.array_equal(mypiv, piv)


def test_triangular_solves_vs_scipy():
    rng = np.random.default_rng(9)
    n = 30
    LU = rng.standard_normal((n, n)) + 5 * np.eye(n)
    B = rng.standard_normal((n, 4))
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    Y = oracle.lu_solve(LU, B)
    ref = sla.solve_triangular(U, sla.solve_triangular(L, B, lower=True, unit_diagonal=True))
    assert np.allclose(Y, ref, rtol=1e-12, atol=1e-12)
    YT = oracle.lu_solve_T(LU, B)
    refT = sla.solve_triangular(L.T, sla.solve_triangular(U.T, B, lower=True), lower=False,
                                unit_diagonal=True)
    assert np.allclose(YT, refT, rtol=1e-12, atol=1e-12)


def test_residual_and_backward_error_formula():
    rng = np.random.default_rng(10)
    A = rng.standard_normal((20, 20))
    X = rng.standard_normal((20, 2))
    B = rng.standard_normal((20, 2))
    R = oracle.residual(A, X, B)
    assert np.allclose(R, B - A @ X, atol=1e-13)
    eta = max(np.abs(B - A @ X)[:, c].max() / (np.abs(A).sum(1).max() * np.abs(X[:, c]).max()
                                                 + np.abs(B[:, c]).max()) for c in range(2))
    assert abs(oracle.backward_error(A, X, B) - eta) <= 1e-12 * eta


# ---------------------------------------------------------------- the method

@pytest.mark.parametrize("kind", [0, 1, 2, 5])
def test_leading_singular_system_solved(kind):
    """The n=256 workload (leading 32 x 32 block of rank 16): without the
    multiplier GENP's growth is catastrophic; with it the solve reaches a
    backward error <= 1e-14 after refinement and the forward error is
    within 1e-14 kappa(A)."""
    A, X, B = (t.numpy() for t in W.lead_deficient(256, 32, 16, 1, 0))
    LU, k = oracle.genp(A)
    growth = np.abs(np.triu(LU)).max() / np.abs(A).max() if k < 0 else np.inf
    plain_eta = oracle.backward_error(A, oracle.lu_solve(LU, B), B) if k < 0 else np.inf
    assert growth > 1e6 or plain_eta > 1e-6
    M = oracle.multiplier(kind, 256, seed=5)
    r = oracle.solve(A, B, M, refine_steps=5, tol=1e-16)
    assert r["step"] == -1
    assert r["eta"][-1] <= 1e-14
    kappa = np.linalg.cond(A, np.inf)
    assert np.abs(r["x"] - X).max() / np.abs(X).max() <= 1e-14 * kappa
    # definition-level result: the GEPP solution
    xd = oracle.gepp_solve(A, B)
    assert np.abs(r["x"] - xd).max() / np.abs(xd).max() <= 1e-14 * kappa


def test_solution_independent_of_multiplier():
    A, X, B = (t.numpy() for t in W.lead_deficient(96, 16, 8, 2, 1))
    xs = [oracle.solve(A, B, oracle.multiplier(0, 96, seed=s), refine_steps=4, tol=1e-17)["x"]
          for s in (1, 2)]
    assert np.abs(xs[0] - xs[1]).max() <= 1e-12 * np.abs(xs[0]).max()


def test_adjoint_vs_finite_differences():
    """dL/dA and dL/dB for L = sum(x^2), x = A^{-1} b at n = 64 in FP64 against
    central differences with h = 1e-6 (relative error <= 1e-6)."""
    n, nrhs = 64, 2
    A, X, B = (t.numpy() for t in W.shifted(1, n, nrhs, 3))
    A, B = A[0], B[0]
    x = oracle.gepp_solve(A, B)
    dA, dB = oracle.adjoint(A, x, 2.0 * x)

    def loss(Am, Bm):
        return float((oracle.gepp_solve(Am, Bm) ** 2).sum())

    rng = np.random.default_rng(0)
    h = 1e-6
    fd, an = [], []
    for _ in range(24):
        i, j = rng.integers(0, n, 2)
        E = np.zeros_like(A)
        E[i, j] = h
        fd.append((loss(A + E, B) - loss(A - E, B)) / (2 * h))
        an.append(dA[i, j])
        c = rng.integers(0, nrhs)
        Eb = np.zeros_like(B)
        Eb[i, c] = h
        fd.append((loss(A, B + Eb) - loss(A, B - Eb)) / (2 * h))
        an.append(dB[i, c])
    fd, an = np.array(fd), np.array(an)
    # relative error of the sampled gradient, normwise (entry-wise it would be
    # dominated by cancellation, eps * loss / h, on the smallest entries)
    assert np.linalg.norm(fd - an) <= 1e-6 * np.linalg.norm(an)


def test_table71_shaped_plausibility():
    """Distribution-level context only (parity with Table 7.1 is unpinned):
    on the paper-shaped n=64 input, GENP without a multiplier is corrupted
    while the circulant-preconditioned solve stays below the paper's worst
    case before refinement."""
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table71.json")))
    worst0 = {row["n"]: row["max"] for row in gold["rows"] if row["iterations"] == 0}
    n = 64
    worse = []
    for seed in range(10):
        A, X, B = (t.numpy() for t in W.table71(n, seed))
        M = oracle.multiplier(1, n, seed=seed)
        r = oracle.solve(A, B, M, refine_steps=0)
        worse.append(oracle.rel_residual_2(A, r["x"], B))
    assert max(worse) <= worst0[n]


# ------------------------------------------------- +-1 circulant multipliers

def test_circulant_pm1_singularity_test_is_exact():
    """For n a power of two every DFT bin of g has power-of-two order, so the
    integer test (sum of g; folded sums for x^m + 1) must agree with the DFT
    computed independently by numpy, on random +-1 vectors and on vectors
    built to vanish at chosen roots of unity."""
    rng = np.random.default_rng(71)
    agree = singular_seen = 0
    for n in (2, 4, 8, 16, 32):
        for _ in range(600):
            g = rng.choice([-1.0, 1.0], n)
            by_fft = np.abs(np.fft.fft(g)).min() < 1e-9
            assert oracle.circulant_pm1_singular(g) == by_fft, (n, g)
            agree += 1
            singular_seen += by_fft
    assert singular_seen > 200            # the singular cases are well represented
    # vanishes at +-i (order 4, x^2 + 1 divides g(x)) but at no other bin
    g = np.array([-1.0, -1.0, -1.0, -1.0, -1.0, 1.0, -1.0, 1.0])
    F = np.abs(np.fft.fft(g))
    assert F[2] < 1e-12 and F[0] > 1 and F[4] > 1 and F[1] > 1
    assert oracle.circulant_pm1_singular(g)
    assert not oracle.circulant_pm1_singular(np.array([1.0, 1.0, 1.0, -1.0]))   # DFT 2, 2j, 2, -2j


def test_circulant_pm1_draws():
    """Entries +-1, the kept draw nonsingular (all DFT bins nonzero), the
    first draw rejected with the frequency of a zero bin (about 0.18 at
    n = 64, Q3), and a redraw only when needed."""
    att = []
    for seed in range(400):
        M = oracle.multiplier(oracle.KIND_CIRCULANT_PM1, 64, seed=seed)
        g = M["g"]
        assert set(np.unique(g)) <= {-1.0, 1.0}
        assert np.abs(np.fft.fft(g)).min() > 1e-6
        att.append(M["attempt"])
    frac = np.mean(np.array(att) > 0)
    assert 0.12 <= frac <= 0.26, frac
    M = oracle.multiplier(oracle.KIND_CIRCULANT_PM1, 1024, seed=3)
    assert np.abs(np.fft.fft(M["g"])).min() > 1e-6


def test_identity_multiplier_is_plain_genp():
    A, _, B = (t.numpy() for t in W.table71(64, seed=2))
    M = oracle.multiplier(oracle.KIND_IDENTITY, 64, seed=0)
    C = oracle.precondition(A, M)
    assert np.array_equal(C, A)
    assert np.array_equal(oracle.apply_multiplier(M, B), B)


# ------------------------------------------------ Toeplitz and Householder

@pytest.mark.parametrize("n", [1, 2, 7, 33])
def test_toeplitz_structure_vs_scipy(n):
    """Definition 3.2 (T_{0,sigma}): the matrix is scipy's Toeplitz matrix of
    its first column t_0 .. t_{n-1} and first row t_0, t_{-1} .. t_{-(n-1)};
    the 2n - 1 draws are distinct."""
    M = oracle.multiplier(5, n, seed=11, scale=0.5)
    t, G = M["t"], M["G"]
    assert t.shape == (2 * n - 1,)
    ref = sla.toeplitz(t[n - 1:], t[n - 1::-1])
    assert np.array_equal(G, ref)
    assert len(np.unique(t)) == 2 * n - 1
    if n > 1:
        assert G[0, n - 1] != G[1, 0]      # not a circulant: the wrap-around entries differ


def test_toeplitz_draws_are_scaled_gaussians():
    n = 20000
    t = oracle.multiplier(5, n, seed=2, scale=3.0)["t"]
    assert abs(t.mean()) < 0.05 * 3.0
    assert abs(t.std() - 3.0) < 0.03 * 3.0
    assert st.kstest(t / 3.0, "norm").pvalue > 1e-3
    t32 = oracle.multiplier(5, 64, seed=2, grid="fp32")["t"]
    assert np.array_equal(t32.astype(np.float32).astype(np.float64), t32)   # on the FP32 grid


def test_toeplitz_products_vs_convolution():
    """(A T)[r][j] = sum_i a_ri t_{i-j}: each row of A T is a slice of the
    full linear correlation of the row with t, computed here by numpy's FFT
    (convolution theorem); x = T y and T^T y likewise."""
    n, m = 48, 5
    rng = np.random.default_rng(4)
    M = oracle.multiplier(5, n, seed=9)
    t = M["t"]
    A = rng.standard_normal((m, n))
    C = oracle.precondition(A, M)
    L = 4 * n
    ft = np.fft.rfft(t, L)
    for r in range(m):
        # sum_i a_i t_{i-j} = sum_i a_i t[i - j + n - 1] = (a reversed * t)[n - 1 - j + (n - 1)]
        full = np.fft.irfft(np.fft.rfft(A[r, ::-1], L) * ft, L)
        ref = np.array([full[(n - 1 - j) + (n - 1)] for j in range(n)])
        assert np.allclose(C[r], ref, rtol=0, atol=1e-12 * np.abs(A[r]).sum() * np.abs(t).max())
    Y = rng.standard_normal((n, 2))
    X = oracle.apply_multiplier(M, Y)
    XT = oracle.apply_multiplier(M, Y, trans=True)
    for c in range(2):
        full = np.fft.irfft(np.fft.rfft(t, L) * np.fft.rfft(Y[:, c], L), L)   # sum_j t[i - j + n - 1] y_j
        assert np.allclose(X[:, c], full[n - 1:2 * n - 1], rtol=0, atol=1e-12 * np.abs(Y).sum() * np.abs(t).max())
        fullT = np.fft.irfft(np.fft.rfft(t[::-1], L) * np.fft.rfft(Y[:, c], L), L)
        assert np.allclose(XT[:, c], fullT[n - 1:2 * n - 1], rtol=0,
                           atol=1e-12 * np.abs(Y).sum() * np.abs(t).max())


@pytest.mark.parametrize("n", [2, 8, 64, 256])
def test_householder_reflector_identities(n):
    """H = I - 2 u u^T / n with u in {+-1}^n: symmetric, H u = -u, H w = w for
    w orthogonal to u, H^2 = I (exact for n a power of two: every entry is
    1 - 2/n or +-2/n), det H = -1."""
    M = oracle.multiplier(6, n, seed=3)
    u, H = M["u"], M["G"]
    assert set(np.unique(u).tolist()) <= {-1.0, 1.0}
    assert np.array_equal(H, H.T)
    assert np.array_equal(H @ u, -u)
    assert np.array_equal(H @ H, np.eye(n))
    w = np.zeros(n)
    i = int(np.argmax(u > 0)) if (u > 0).any() else 0
    j = int(np.argmax(u < 0)) if (u < 0).any() else 1
    if u[i] != u[j]:
        w[i], w[j] = 1.0, 1.0            # u^T w = 0
        assert np.array_equal(H @ w, w)
    sign, logdet = np.linalg.slogdet(H)
    assert sign == -1.0 and abs(logdet) < 1e-12
    assert np.array_equal(oracle.precondition(np.eye(n), M), H)
    assert np.array_equal(oracle.apply_multiplier(M, np.eye(n), trans=True), H)


def test_householder_signs_balanced():
    u = oracle.multiplier(6, 100000, seed=1)["u"]
    assert abs(u.mean()) < 0.02


def test_householder_repairs_rank_one_deficiency_only():
    """A H = A - (2/n)(A u) u^T changes A by rank one.  On the paper-shaped
    inputs (leading n/2 x n/2 block of numerical rank n/2 - 1, the kind of
    matrices the cited Householder tests used) it repairs GENP and the solve
    reaches eta <= 1e-14; on the workload whose leading 32 x 32 block has
    rank 16 no rank-one change can, and the growth stays catastrophic."""
    A, X, B = (t.numpy() for t in W.table71(128, 3))
    LU0, k0 = oracle.genp(A)
    plain = oracle.backward_error(A, oracle.lu_solve(LU0, B), B) if k0 < 0 else np.inf
    M = oracle.multiplier(6, 128, seed=5)
    r = oracle.solve(A, B, M, refine_steps=5, tol=1e-16)
    assert r["step"] == -1
    assert r["eta"][-1] <= 1e-14
    assert r["eta"][0] < plain / 100
    xd = oracle.gepp_solve(A, B)
    assert np.abs(r["x"] - xd).max() / np.abs(xd).max() <= 1e-14 * np.linalg.cond(A, np.inf)
    A2, _, _ = (t.numpy() for t in W.lead_deficient(256, 32, 16, 1, 0))
    LU, k = oracle.genp(oracle.precondition(A2, oracle.multiplier(6, 256, seed=5)))
    assert k >= 0 or np.abs(np.triu(LU)).max() / np.abs(A2).max() > 1e10


# ------------------------------------------------ the left multiplier (G A)

@pytest.mark.parametrize("kind", [0, 1, 2, 5])
def test_left_multiplier_solves_leading_singular_system(kind):
    """The GM half of Cor. 4.1: the leading blocks of G A are nonsingular
    w.p. 1, so GENP of C = G A is safe on the rank-16 workload; x solves
    A x = b because G A x = G b; refinement reaches eta <= 1e-14 and the
    GEPP solution within 1e-14 kappa."""
    A, X, B = (t.numpy() for t in W.lead_deficient(256, 32, 16, 1, 0))
    M = oracle.multiplier(kind, 256, seed=5)
    C = oracle.precondition_left(A, M)
    assert np.array_equal(C, oracle.matmul(M["G"], A))
    r = oracle.solve(A, B, M, refine_steps=5, tol=1e-16, side="left")
    assert r["step"] == -1
    assert r["eta"][-1] <= 1e-14
    kappa = np.linalg.cond(A, np.inf)
    xd = oracle.gepp_solve(A, B)
    assert np.abs(r["x"] - xd).max() / np.abs(xd).max() <= 1e-14 * kappa


def test_left_multiplier_leading_minors_by_leibniz():
    """Every leading minor of G A is nonzero (checked exactly, in rationals)
    on a nonsingular 5 x 5 A whose leading 1 x 1 and 2 x 2 blocks are
    singular: plain GENP breaks down, GENP of G A does not, and the product
    of its pivots is det(G A) = det(G) det(A)."""
    A = np.array([[0., 2., 0., 1., 3.], [0., 4., 1., 0., 1.], [0., 1., 5., 2., 2.], [1., 0., 2., 3., 1.],
                  [3., 1., 1., 1., 4.]])
    assert oracle.det_leibniz(A[:1, :1]) == 0 and oracle.det_leibniz(A[:2, :2]) == 0
    assert oracle.det_leibniz(A) != 0
    assert oracle.genp(A)[1] == 0
    M = oracle.multiplier(0, 5, seed=3)
    C = oracle.precondition_left(A, M)
    for k in range(1, 6):
        assert oracle.det_leibniz(C[:k, :k]) != 0
    LU, step = oracle.genp(C)
    assert step == -1
    prod = float(np.prod(np.diag(LU)))
    ref = float(oracle.det_leibniz(M["G"]) * oracle.det_leibniz(A))
    assert abs(prod - ref) <= 1e-12 * abs(ref)


# ------------------------------------------------ low-rank approximation (Sec. 5)

def test_sketch_multiplier_structure():
    G = oracle.sketch_multiplier(50, 8, seed=3)
    assert G.shape == (50, 8) and len(np.unique(G)) == 400
    T = oracle.sketch_multiplier(50, 8, seed=3, toeplitz=True)
    for i in range(1, 50):
        for j in range(1, 8):
            assert T[i, j] == T[i - 1, j - 1]               # constant along diagonals
    g = oracle.sketch_multiplier(4000, 5, seed=1).ravel()
    assert abs(g.mean()) < 0.03 and abs(g.std() - 1.0) < 0.03


@pytest.mark.parametrize("n,q", [(64, 1), (128, 8), (256, 32)])
def test_lowrank_exact_rank_is_recovered(n, q):
    """With an exactly rank-q A (tail singular values 0) the sketch A^T G
    spans A's row space w.p. 1, so A Q Q^T reproduces A to rounding, and
    B Y reproduces the leading right singular vectors (Thm. 5.1 with no
    perturbation)."""
    A, S, T, s = (t.numpy() for t in W.lowrank(n, q, seed=2))
    A = (S[:, :q] * s[:q]) @ T[:, :q].T
    r = oracle.lowrank_approx(A, oracle.sketch_multiplier(n, q, seed=5))
    assert np.allclose(r["Q"].T @ r["Q"], np.eye(q), atol=1e-13)
    rn1, rn2 = oracle.lowrank_residuals(A, r["B"], r["Q"], r["AQ"], T[:, :q])
    assert rn2 <= 1e-13 and rn1 <= 1e-10


@pytest.mark.parametrize("toeplitz", [False, True])
def test_lowrank_residual_between_eckart_young_and_tail_bound(toeplitz):
    """For the Table 7.2 / 7.3 inputs (sigma_{q+1} = 1e-10) every rank-q
    approximation errs by at least sigma_{q+1} (Eckart-Young), and the
    randomized one stays within a modest factor of it (Sec. 5, the paper's
    observed 1e-9 .. 1e-6)."""
    n, q = 128, 8
    A, S, T, s = (t.numpy() for t in W.lowrank(n, q, seed=4))
    assert abs(np.linalg.norm(A, 2) - 1.0) < 1e-12
    r = oracle.lowrank_approx(A, oracle.sketch_multiplier(n, q, seed=9, toeplitz=toeplitz))
    rn1, rn2 = oracle.lowrank_residuals(A, r["B"], r["Q"], r["AQ"], T[:, :q])
    assert 1e-10 * (1 - 1e-6) <= rn2 <= 1e-5
    assert rn1 <= 1e-4
    # Q is the QR factor with a positive diagonal: B = Q R, R upper triangular
    R = r["Q"].T @ r["B"]
    assert np.allclose(np.tril(R, -1), 0.0, atol=1e-12 * np.abs(R).max())
    assert np.all(np.diag(R) > 0)
    assert np.allclose(r["Q"] @ R, r["B"], atol=1e-13 * np.abs(r["B"]).max())


# ------------------------------------------------ numerical rank (App. B)

@pytest.mark.parametrize("n,q,seed", [(64, 1, 0), (64, 8, 1), (128, 8, 2), (128, 32, 3), (256, 32, 4), (256, 17, 5)])
def test_numerical_rank_of_tables_inputs(n, q, seed):
    """Inputs with numerical rank q (s_j = 1/j up to q, 1e-10 beyond): the
    binary search returns q from the full range [0, min(n, 128)], its trace
    is consistent (every r <= q passed, every r > q failed), and the basis
    is A^T G_q."""
    A, S, T, s = (t.numpy() for t in W.lowrank(n, q, seed))
    G = oracle.sketch_multiplier(n, min(n, 128), seed=seed + 7)
    rank, B, trace = oracle.numerical_rank(A, 0, min(n, 128), 1e6, G)
    assert rank == q
    for r, kappa, ok in trace:
        assert ok == (r <= q)
    assert np.array_equal(B, oracle.matmul(A.T.copy(), G[:, :q].copy()))
    # the basis spans the leading right singular space (Thm. 5.1): sine of the largest angle small
    Qb = np.linalg.qr(B)[0]
    assert np.linalg.norm(T[:, :q] - Qb @ (Qb.T @ T[:, :q]), 2) <= 1e-5      # the tables: rn1 up to ~1e-5


def test_numerical_rank_degenerate_ranges():
    A, S, T, s = (t.numpy() for t in W.lowrank(64, 8, 0))
    G = oracle.sketch_multiplier(64, 32, seed=1)
    assert oracle.numerical_rank(A, 5, 5, 1e6, G)[0] == 5          # r_lo = r_hi: no test
    assert oracle.numerical_rank(A, 0, 4, 1e6, G)[0] == 4          # rank above the range: r_hi
    assert oracle.numerical_rank(A, 12, 32, 1e6, G)[0] == 12       # rank below the range: r_lo


# --------------------------------------------------------------------------
# Fixed-point grid of the sliced product
# --------------------------------------------------------------------------

def _balanced_digits(X, nd):
    """Balanced base-128 digits of integers X (most significant first), by
    Python integer arithmetic: X = sum_t d_t 128^(nd-1-t)."""
    out = []
    for x in X:
        x = int(x)
        ds = []
        for _ in range(nd - 1):
            lo = ((x + 64) % 128) - 64
            ds.append(lo)
            x = (x - lo) // 128
        ds.append(x)
        out.append(ds[::-1])
    return np.array(out)


@pytest.mark.parametrize("n", [64, 300, 1024])
def test_sliced_grid_exact_in_two_digits(n):
    """Every column of the gridded Gaussian, scaled by its own power of two
    2^-f (f the least with max |g| < 2^f) and by 2^14, is an integer below
    2^14 in magnitude, and two balanced 7-bit digits rebuild it exactly
    (|d_1| <= 128, |d_2| <= 64): the two-digit slicing loses nothing."""
    s = 1.0 / math.sqrt(n)
    G = oracle.sliced_grid(oracle.multiplier(0, n, seed=n, grid="fp32")["G"], s)
    for j in range(n):
        col = G[:, j]
        f = math.frexp(float(np.abs(col).max()))[1]
        X = np.ldexp(col, 14 - f)
        assert np.array_equal(X, np.round(X))
        assert np.abs(X).max() < 2**14
        d = _balanced_digits(X, 2)
        assert np.abs(d[:, 0]).max() <= 128 and np.abs(d[:, 1]).max() <= 64
        assert np.array_equal(d[:, 0] * 128 + d[:, 1], X.astype(np.int64))


@pytest.mark.parametrize("n", [64, 300, 1024])
def test_sliced_grid_exact_in_one_digit(n):
    """The one-digit grid: every column scaled by its own power of two 2^-f
    (f the least with max |g| < 2^f) and by 2^7 is an integer below 2^7 in
    magnitude, so one balanced digit (|d_1| <= 128) holds it exactly; the
    grid is the two-digit grid's coarsening (every one-digit value is a
    two-digit value) and moves an entry by at most 2^(E - 7)."""
    s = 1.0 / math.sqrt(n)
    G0 = oracle.multiplier(0, n, seed=n, grid="fp32")["G"]
    G = oracle.sliced_grid(G0, s, digits=1)
    E = oracle.sliced_grid_exponent(s)
    assert np.abs(G - G0).max() <= 2.0 ** (E - 7)
    assert np.array_equal(oracle.sliced_grid(G, s, digits=2), G)
    for j in range(n):
        col = G[:, j]
        amax = float(np.abs(col).max())
        if amax == 0.0:
            continue
        f = math.frexp(amax)[1]
        X = np.ldexp(col, 7 - f)
        assert np.array_equal(X, np.round(X))
        assert np.abs(X).max() < 2**7


def test_sliced_grid_one_digit_rounding():
    """Nearest multiple of 2^(E - 6), ties to even, by hand; the coarser grid
    keeps the Gaussian's first two moments within 1%."""
    n = 512
    s = 1.0 / math.sqrt(n)
    q = 2.0 ** (oracle.sliced_grid_exponent(s) - 6)
    T = np.array([[0.5 * q, 1.5 * q, 2.5 * q, -0.5 * q, -1.5 * q, 0.49 * q]])
    assert np.array_equal(oracle.sliced_grid(T, s, digits=1) / q, [[0.0, 2.0, 2.0, -0.0, -2.0, 0.0]])
    G = oracle.sliced_grid(oracle.multiplier(0, n, seed=3)["G"], s, digits=1)
    assert np.array_equal(G / q, np.round(G / q))
    assert abs(G.std() / s - 1) < 0.01 and abs(G.mean()) < 0.01 * s
    with pytest.raises(ValueError):
        oracle.sliced_grid(G, s, digits=3)


def test_sliced_grid_rounding_and_exponent():
    """E is the least integer with 12.5 scale <= 2^E; entries move to the
    nearest multiple of 2^(E-13) (error <= 2^(E-14)), ties to even; the grid
    keeps the Gaussian's moments (a perturbation of at most 1.6e-3 scale)."""
    for scale in (1.0, 1 / 64, 1 / math.sqrt(300), 0.08, 12.5 ** -1, 3.0):
        E = oracle.sliced_grid_exponent(scale)
        assert 12.5 * scale <= 2.0 ** E and 12.5 * scale > 2.0 ** (E - 1)
    n = 512
    s = 1.0 / math.sqrt(n)
    G0 = oracle.multiplier(0, n, seed=3)["G"]
    G = oracle.sliced_grid(G0, s)
    q = 2.0 ** (oracle.sliced_grid_exponent(s) - 13)
    assert np.abs(G - G0).max() <= q / 2
    assert np.array_equal(G / q, np.round(G / q))
    assert abs(G.std() / s - 1) < 0.01 and abs(G.mean()) < 0.01 * s
    # ties to even, by hand
    T = np.array([[0.5 * q, 1.5 * q, 2.5 * q, -0.5 * q, -1.5 * q]])
    assert np.array_equal(oracle.sliced_grid(T, s) / q, [[0.0, 2.0, 2.0, -0.0, -2.0]])


# --------------------------------------------------------------------------
# Block Gaussian elimination with explicit pivot-block inverses (Sec. 2,
# Theorem 2.2's block form)
# --------------------------------------------------------------------------

def _unimodular(rng, k):
    """An integer k x k matrix L0 U0 (unit lower times upper with +-1
    diagonal, small entries): nonsingular leading minors, integer inverse."""
    L0 = np.tril(rng.integers(-1, 2, (k, k)), -1) + np.eye(k, dtype=np.int64)
    U0 = np.triu(rng.integers(-1, 2, (k, k)), 1) + np.diag(rng.choice([-1, 1], k))
    return L0 @ U0


def _exact_inverse(M):
    """Inverse of an integer matrix in exact rationals (Gauss-Jordan with
    row exchanges on Fractions: a different algorithm from the oracle's)."""
    k = len(M)
    A = [[Fraction(int(M[i][j])) for j in range(k)] + [Fraction(int(i == j)) for j in range(k)] for i in range(k)]
    for c in range(k):
        p = next(r for r in range(c, k) if A[r][c] != 0)
        A[c], A[p] = A[p], A[c]
        piv = A[c][c]
        A[c] = [v / piv for v in A[c]]
        for r in range(k):
            if r != c and A[r][c] != 0:
                f = A[r][c]
                A[r] = [a - f * b for a, b in zip(A[r], A[c])]
    return [[A[i][k + j] for j in range(k)] for i in range(k)]


@pytest.mark.parametrize("k", [1, 2, 5, 9])
def test_gauss_jordan_inverse_exact_on_unimodular(k):
    rng = np.random.default_rng(40 + k)
    P = _unimodular(rng, k)
    X, t = oracle.gauss_jordan_inverse(P.astype(float))
    assert t == -1
    ref = _exact_inverse(P)
    assert all(X[i, j] == float(ref[i][j]) for i in range(k) for j in range(k))
    assert np.array_equal(X @ P, np.eye(k))


def test_gauss_jordan_inverse_vs_lapack_and_breakdown():
    rng = np.random.default_rng(3)
    P = rng.standard_normal((40, 40)) + 8 * np.eye(40)
    X, t = oracle.gauss_jordan_inverse(P)
    assert t == -1
    ref = np.linalg.inv(P)
    assert np.abs(X - ref).max() <= 40 * 2.0**-52 * np.linalg.cond(P) * np.abs(ref).max()
    _, t = oracle.gauss_jordan_inverse(np.array([[0.0, 1.0], [1.0, 0.0]]))
    assert t == 0                                   # singular leading 1 x 1 minor
    _, t = oracle.gauss_jordan_inverse(np.array([[1.0, 2.0, 0.0], [2.0, 4.0, 1.0], [0.0, 1.0, 1.0]]))
    assert t == 1                                   # singular leading 2 x 2 minor


@pytest.mark.parametrize("n,nb", [(12, 3), (13, 4), (20, 7)])
def test_block_genp_recovers_integer_block_factors(n, nb):
    """C = L0 D U0 with L0 block unit lower and U0 block unit upper integer
    matrices (identity diagonal blocks) and D block diagonal with unimodular
    integer blocks: every step is exact, so block GE returns L_B = L0, the
    pivot blocks P_k = D_k, the block row U_kj = D_k U0_kj and P_k^{-1} equal
    to the exact rational inverse of D_k, bit for bit (ragged last block
    included)."""
    rng = np.random.default_rng(n * 31 + nb)
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
    C = (L0 @ D @ U0).astype(float)
    LU, Pinv, k = oracle.block_genp(C, nb)
    assert k == -1
    DU = D @ U0
    for bi, (a, b) in enumerate(blocks):
        for bj, (c, d) in enumerate(blocks):
            want = L0[a:b, c:d] if bj < bi else DU[a:b, c:d]
            assert np.array_equal(LU[a:b, c:d], want.astype(float))
        ref = _exact_inverse(D[a:b, a:b])
        kb = b - a
        assert all(Pinv[bi][i, j] == float(ref[i][j]) for i in range(kb) for j in range(kb))


def test_block_genp_schur_complement_in_rationals():
    """The second pivot block of block GE with nb = 3 on a 6 x 6 integer C is
    the Schur complement C22 - C21 C11^{-1} C12 (Fact 2.1), here computed in
    exact rationals; the first is C11 itself; det C = det P_0 det P_1
    (Leibniz expansions in rationals)."""
    rng = np.random.default_rng(8)
    while True:
        C = rng.integers(-5, 6, (6, 6)).astype(float)
        if oracle.det_leibniz(C[:3, :3]) != 0 and oracle.det_leibniz(C) != 0:
            break
    LU, Pinv, k = oracle.block_genp(C, 3)
    assert k == -1
    assert np.array_equal(LU[:3, :3], C[:3, :3])
    Ci = _exact_inverse(C[:3, :3])
    S = [[Fraction(int(C[3 + i, 3 + j])) - sum(Fraction(int(C[3 + i, p])) * Ci[p][q] * Fraction(int(C[q, 3 + j]))
                                               for p in range(3) for q in range(3))
          for j in range(3)] for i in range(3)]
    for i in range(3):
        for j in range(3):
            assert abs(LU[3 + i, 3 + j] - float(S[i][j])) <= 1e-13 * max(1.0, abs(float(S[i][j])))
    dP1 = oracle.det_leibniz(np.array([[float(S[i][j]) for j in range(3)] for i in range(3)]))
    assert abs(float(oracle.det_leibniz(C[:3, :3]) * dP1) - float(oracle.det_leibniz(C))) <= \
        1e-10 * abs(float(oracle.det_leibniz(C)))


def test_block_genp_nb1_is_genp_and_pivot_blocks_are_LkkUkk():
    """nb = 1 is GENP (multiplying by the reciprocal pivot instead of
    dividing: within one rounding per entry); for nb = 16 every pivot block
    equals L_kk U_kk of GENP's factors (the leading block of the Schur
    complement), and L_B = L diag(L_kk^{-1})."""
    A, _, _ = W.lead_deficient(64, 8, 4, 1, 2)
    C = oracle.precondition(A.numpy(), oracle.multiplier(0, 64, seed=3))
    LUp, k = oracle.genp(C)
    assert k == -1
    LU1, P1, k1 = oracle.block_genp(C, 1)
    assert k1 == -1
    assert np.abs(LU1 - LUp).max() <= 1e-12 * np.abs(LUp).max()
    LU16, P16, k16 = oracle.block_genp(C, 16)
    L, U = oracle.split_lu(LUp)
    for b in range(4):
        s = slice(16 * b, 16 * b + 16)
        Pk = L[s, s] @ U[s, s]
        assert np.abs(LU16[s, s] - Pk).max() <= 1e-12 * np.abs(Pk).max()
        assert np.abs(P16[b] @ LU16[s, s] - np.eye(16)).max() <= 1e-10
        for b2 in range(b + 1, 4):
            s2 = slice(16 * b2, 16 * b2 + 16)
            want = L[s2, s] @ np.linalg.inv(L[s, s])
            assert np.abs(LU16[s2, s] - want).max() <= 1e-10 * max(1.0, np.abs(want).max())


def test_thm22_block_pivot_bounds():
    """Thm. 2.2, block form: every pivot block has ||P_k|| <= N + N_- N^2 and
    ||P_k^{-1}|| <= N_-, N = ||C||, N_- = max_j ||(C_j^(j))^{-1}|| (2-norms,
    leading blocks by brute force)."""
    for seed in range(3):
        A, _, _ = W.lead_deficient(96, 16, 8, 1, seed)
        C = oracle.precondition(A.numpy(), oracle.multiplier(0, 96, seed=seed))
        N = np.linalg.norm(C, 2)
        Nm = max(np.linalg.norm(np.linalg.inv(C[:j, :j]), 2) for j in range(1, 97))
        LU, Pinv, k = oracle.block_genp(C, 16)
        assert k == -1
        for b in range(6):
            s = slice(16 * b, 16 * b + 16)
            assert np.linalg.norm(LU[s, s], 2) <= (N + Nm * N * N) * (1 + 1e-10)
            assert np.linalg.norm(Pinv[b], 2) <= Nm * (1 + 1e-8)


@pytest.mark.parametrize("nb", [16, 32, 48])
def test_block_genp_solves_leading_singular_system(nb):
    """The n = 256 workload (leading 32 x 32 block of rank 16): block GE of
    A itself fails (the first pivot block is singular to working precision),
    block GE of A G with a Gaussian multiplier reaches eta <= 1e-14 after
    refinement and the GEPP solution within 1e-14 kappa(A)."""
    A, X, B = (t.numpy() for t in W.lead_deficient(256, 32, 16, 1, 0))
    LU, Pinv, k = oracle.block_genp(A, 32)
    if k < 0:
        plain = oracle.block_lu_solve(LU, Pinv, 32, B)
        assert not np.all(np.isfinite(plain)) or oracle.backward_error(A, plain, B) > 1e-8
    M = oracle.multiplier(0, 256, seed=5)
    r = oracle.block_solve(A, B, M, nb, refine_steps=5, tol=1e-16)
    assert r["step"] == -1
    assert r["eta"][-1] <= 1e-14
    kappa = np.linalg.cond(A, np.inf)
    xd = oracle.gepp_solve(A, B)
    assert np.abs(r["x"] - xd).max() / np.abs(xd).max() <= 1e-14 * kappa
    assert np.abs(r["x"] - X).max() / np.abs(X).max() <= 1e-14 * kappa


# --------------------------------------------------------------------------
# FP8 (e4m3) operands with per-tile power-of-two scales
# --------------------------------------------------------------------------

def _torch_e4m3():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8_e4m3fn")
    return torch


def test_e4m3_decode_matches_torch():
    """All 256 codes against PyTorch's float8_e4m3fn (an independent
    implementation of the same format): equal values, the same two NaNs."""
    torch = _torch_e4m3()
    codes = np.arange(256, dtype=np.uint8)
    v = oracle.e4m3_decode(codes)
    t = torch.tensor(codes).view(torch.float8_e4m3fn).double().numpy()
    assert np.array_equal(np.isnan(v), np.isnan(t)) and int(np.isnan(v).sum()) == 2
    assert np.array_equal(v[~np.isnan(v)], t[~np.isnan(t)])
    assert v[0x7E] == 448.0 and v[0x01] == 2.0 ** -9 and v[0x08] == 2.0 ** -6
    fin = ~np.isnan(v)
    assert np.array_equal(oracle.e4m3_encode(v[fin]), codes[fin])


def test_e4m3_round_matches_torch_and_brute_force():
    """Rounding to nearest, ties to even: against PyTorch's float32 ->
    float8_e4m3fn conversion on random values and on every midpoint between
    neighbouring grid values (inside the finite range, where its rule agrees),
    and against a brute-force nearest-grid-value search."""
    torch = _torch_e4m3()
    rng = np.random.default_rng(7)
    x = rng.standard_normal(100000) * np.exp2(rng.uniform(-14, 9, 100000))
    x = x.astype(np.float32).astype(np.float64)
    x = x[np.abs(x) < 448.0]
    r = oracle.e4m3_round(x)
    t = torch.tensor(x, dtype=torch.float32).to(torch.float8_e4m3fn).double().numpy()
    assert np.array_equal(r, t)
    grid = oracle.e4m3_decode(np.arange(256, dtype=np.uint8))
    pos = np.unique(grid[np.isfinite(grid) & (grid >= 0)])
    mid = (pos[:-1] + pos[1:]) / 2
    rm = oracle.e4m3_round(mid)
    tm = torch.tensor(mid, dtype=torch.float32).to(torch.float8_e4m3fn).double().numpy()
    assert np.array_equal(rm, tm)
    # ties go to the neighbour with the even code
    codes = oracle.e4m3_encode(rm)
    assert np.all(codes % 2 == 0)
    # brute force on a sample: the nearest grid value, ties to the even code
    for v in np.concatenate([x[:2000], mid]):
        d = np.abs(pos - abs(v))
        best = np.flatnonzero(d == d.min())
        pick = pos[best[0]] if len(best) == 1 else [g for g in pos[best] if oracle.e4m3_encode(g) % 2 == 0][0]
        assert oracle.e4m3_round(v) == math.copysign(pick, v)


def test_e4m3_saturates_at_448():
    x = np.array([448.0, 463.99, 464.0, 480.0, 1e6, -1e30])
    assert np.array_equal(oracle.e4m3_round(x), np.array([448.0, 448.0, 448.0, 448.0, 448.0, -448.0]))


def test_tile_exponent_is_the_least_that_fits():
    """2^e is the smallest power of two with amax <= 448 2^e."""
    rng = np.random.default_rng(3)
    amaxes = np.concatenate([np.exp2(rng.uniform(-100, 100, 2000)),
                             448.0 * np.exp2(np.arange(-20, 21)),
                             np.nextafter(448.0 * np.exp2(np.arange(-20, 21)), np.inf),
                             np.nextafter(448.0 * np.exp2(np.arange(-20, 21)), 0.0)])
    for a in amaxes:
        e = oracle.tile_exponent(a)
        assert a <= 448.0 * 2.0 ** e
        assert a > 448.0 * 2.0 ** (e - 1)
    assert oracle.tile_exponent(0.0) == 0
    assert oracle.tile_exponent(1e-300) == -126 and oracle.tile_exponent(1e300) == 126


def test_quantize_e4m3_error_bounds_and_tiles():
    """Every tile: |x - dequantized| <= 2^-4 |x| where the code is normal,
    <= 2^-10 s where it is subnormal (s the tile's scale); the tile maximum
    lands in [224, 448]; a zero tile gets scale 1 and zero codes."""
    rng = np.random.default_rng(11)
    m, K = 300, 270
    X = rng.standard_normal((m, K)) * np.exp2(rng.uniform(-20, 20, (m, 1)))
    X[128:256, 128:256] = 0.0
    codes, scales = oracle.quantize_e4m3(X)
    assert scales.shape == (3, 3) and codes.shape == (m, K)
    D = oracle.dequantize_e4m3(codes, scales)
    S = np.repeat(np.repeat(scales, 128, 0), 128, 1)[:m, :K]
    sub = np.abs(X / S) < 2.0 ** -6
    assert np.all(np.abs(D - X)[~sub] <= 2.0 ** -4 * np.abs(X)[~sub])
    assert np.all(np.abs(D - X)[sub] <= 2.0 ** -10 * S[sub])
    assert scales[1, 1] == 1.0 and not codes[128:256, 128:256].any()
    for ti in range(3):
        for kt in range(3):
            blk = np.abs(X[ti * 128:(ti + 1) * 128, kt * 128:(kt + 1) * 128]) / scales[ti, kt]
            if blk.max() > 0:
                assert 224.0 < blk.max() <= 448.0


def test_gemm_e4m3_exact_on_small_integers():
    """Integers of magnitude <= 15 are exact e4m3 values at every tile scale
    the rule picks (4 significant bits), so the tile-scaled product must equal
    the integer product exactly, over several k-tiles and ragged edges."""
    rng = np.random.default_rng(5)
    m, n, K = 200, 150, 333
    A = rng.integers(-15, 16, (m, K))
    B = rng.integers(-15, 16, (K, n))
    A[:128, :128] = rng.integers(-3, 4, (128, 128))          # another tile scale
    Aq, sA = oracle.quantize_e4m3(A.astype(np.float64))
    Bq, sB = oracle.quantize_e4m3(B.T.astype(np.float64))
    assert np.array_equal(oracle.dequantize_e4m3(Aq, sA), A)
    D = oracle.gemm_e4m3(Aq, sA, Bq, sB, alpha=2.0, beta=-1.0, C=np.ones((m, n)))
    assert np.array_equal(D, 2.0 * (A @ B).astype(np.float64) - 1.0)


def test_fp8_grid_multiplier():
    """The FP8 grid: one exponent e for the matrix with 12.5 scale <= 448 2^e
    (the polar method never draws beyond 12.1 standard deviations, so nothing
    saturates), every entry an e4m3 value times 2^e, the nearest one."""
    n = 256
    M = oracle.multiplier(oracle.KIND_GAUSSIAN, n, seed=4, grid="fp32")
    s = 1.0 / np.sqrt(n)
    G8 = oracle.fp8_grid(M["G"], s)
    e = oracle.tile_exponent(12.5 * s)
    assert 12.5 * s <= 448.0 * 2.0 ** e < 2 * 12.5 * s
    q = np.ldexp(G8, -e)
    assert np.array_equal(oracle.e4m3_round(q), q)
    assert np.max(np.abs(q)) < 448.0
    rel = np.abs(G8 - M["G"]) / np.abs(M["G"])
    big = np.abs(q) >= 2.0 ** -6
    assert np.all(rel[big] <= 2.0 ** -4)


def test_genp_fp8_is_genp_below_one_block():
    """n <= nb: no Schur update, so the FP8 blocked GENP is plain GENP."""
    A = np.random.default_rng(1).standard_normal((100, 100)) + 20 * np.eye(100)
    LU1, s1 = oracle.genp(A)
    LU2, s2 = oracle.genp_fp8(A)
    assert np.array_equal(LU1, LU2) and s1 == s2 == -1


def test_genp_fp8_recovers_small_integer_factors_exactly():
    """C = L0 U0 with small integer factors: every Schur complement is an
    integer, and the block row and column (entries of L0 and U0, magnitude
    <= 3) are exact e4m3 values at every tile scale, so the e4m3 Schur
    products are exact and the blocked factorization returns L0 and U0 bit
    for bit (a transposed operand, a wrong tile or a wrong scale would not)."""
    rng = np.random.default_rng(8)
    n = 300
    L0 = np.tril(rng.integers(-2, 3, (n, n)), -1) + np.eye(n)
    U0 = np.triu(rng.integers(-3, 4, (n, n)), 1) + np.diag(rng.choice([-1.0, 1.0, 2.0], n))
    LU, step = oracle.genp_fp8(L0 @ U0, nb=128)
    assert step == -1
    assert np.array_equal(np.tril(LU, -1) + np.eye(n), L0) and np.array_equal(np.triu(LU), U0)


def test_genp_fp8_backward_error_bound():
    """Gaussian data: |L U - C| <= (2^-3 + 2^-7) |L||U| (two e4m3 roundings of
    2^-4 per Schur product) plus the subnormal codes' absolute error, and the
    error is genuinely 8-bit (above 1e-3 relative somewhere)."""
    n = 384
    A, _, _ = W.lead_deficient(n, 16, 8, 1, seed=3)
    C = oracle.precondition(A.numpy(), oracle.multiplier(0, n, seed=5))
    LU, step = oracle.genp_fp8(C)
    assert step == -1
    L, U = oracle.split_lu(LU)
    E = np.abs(L @ U - C)
    B = np.abs(L) @ np.abs(U)
    sub = 2 * 2.0 ** -10 / 224 * np.max(np.abs(L)) * np.max(np.abs(U)) * n
    assert np.all(E <= (2.0 ** -3 + 2.0 ** -7) * B + sub)
    assert np.max(E / np.maximum(B, 1e-300)) > 1e-3


def test_fp8_factors_precondition_only_at_small_growth():
    """The FP8 reading: with growth ~1 (plain GENP of a Gaussian matrix with a
    0.1 n diagonal shift) e4m3 factors drive classic FP64 refinement to
    eta <= 1e-14; the same matrix times a Gaussian multiplier has growth
    ~1e5, and the refinement does not move eta off ~0.1."""
    n = 512
    A, _, B = (t.numpy() for t in W.shifted(1, n, 2, seed=4))
    A, B = A[0], B[0]
    LU, _ = oracle.genp_fp8(A)
    X = oracle.lu_solve(LU, B)
    for _ in range(8):
        X = X + oracle.lu_solve(LU, oracle.residual(A, X, B))
    assert oracle.backward_error(A, X, B) <= 1e-14
    M = oracle.multiplier(0, n, seed=3)
    C = oracle.precondition(A, M)
    LU, _ = oracle.genp_fp8(C)
    assert np.abs(np.triu(LU)).max() / np.abs(C).max() > 1e4
    X = oracle.apply_multiplier(M, oracle.lu_solve(LU, B))
    for _ in range(8):
        X = X + oracle.apply_multiplier(M, oracle.lu_solve(LU, oracle.residual(A, X, B)))
    assert oracle.backward_error(A, X, B) > 1e-2
