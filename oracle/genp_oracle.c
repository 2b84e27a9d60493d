/*
 * genp_oracle.c -- plain, slow CPU FP64 oracle for randomized GENP.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant generator with the CUDA library, and the
 * CUDA library never calls it.
 *
 * Every routine is the textbook definition written out with plain loops, in
 * IEEE double, compiled with -ffp-contract=off so that no multiply-add is
 * fused behind our back (the random-number routines must reproduce the
 * CUDA path bit for bit; everything else is compared with tolerances).
 *
 * Storage: row-major with an explicit leading dimension, a[i*lda + j].
 *
 * Method (Pan & Qian, "More on the Power of Randomized Matrix
 * Multiplication", Sec. 1.1 and Cor. 4.1): pick a random multiplier G,
 * form C = A*G, run Gaussian elimination with no pivoting on C, solve
 * L*U*y = b and return x = G*y.  Theorem 4.1 (the MH form, M = A, H = G)
 * and Corollary 4.1 state that every leading block of A*G is as well
 * conditioned as A up to a modest random factor, which is what makes GENP
 * on C numerically safe.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* Counter-based generator: Philox4x64-10 (Salmon, Moraes, Dror, Shaw,       */
/* "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11, Sec. 3.3).  Each    */
/* round multiplies words 0 and 2 by two fixed odd constants, keeps the high */
/* and low halves of the 128-bit products, xors the high halves with the     */
/* other two words and the round key, and permutes; the key is bumped by two */
/* Weyl constants between rounds.                                            */
/* ------------------------------------------------------------------------ */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

OR_EXPORT void or_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2],
                                uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, c0, &hi0, &lo0);
        mulhilo64(M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 53 random bits -> [0, 1), exact. */
OR_EXPORT double or_u53(uint64_t w) { return (double)(w >> 11) * 0x1.0p-53; }

/* Natural log for a positive normal double, from the atanh series
 * ln(m) = 2 atanh((m-1)/(m+1)) = 2 (f + f^3/3 + f^5/5 + ...)
 * (Abramowitz & Stegun 4.1.27) after the exact split s = m * 2^e with
 * m in (sqrt(2)/2, sqrt(2)].  |f| <= 0.1716, so f^2 <= 0.0295 and twelve
 * terms push the truncation below 2^-60.  Only +, -, *, / are used. */
OR_EXPORT double or_log(double s) {
    uint64_t b;
    memcpy(&b, &s, 8);
    int e = (int)((b >> 52) & 0x7ff) - 1023;
    uint64_t mb = (b & 0x000FFFFFFFFFFFFFULL) | (1023ULL << 52);
    double m;
    memcpy(&m, &mb, 8);                       /* m in [1, 2) */
    const double SQRT2 = 1.4142135623730951;  /* nearest double to sqrt(2) */
    const double LN2 = 0.6931471805599453;    /* nearest double to ln(2)   */
    if (m > SQRT2) { m = m * 0.5; e = e + 1; }
    double f = (m - 1.0) / (m + 1.0);
    double f2 = f * f;
    const int K = 11;
    double p = 1.0 / (double)(2 * K + 1);
    for (int k = K - 1; k >= 0; --k) {
        double t = p * f2;
        p = t + 1.0 / (double)(2 * k + 1);
    }
    double tf = 2.0 * f;
    double lm = tf * p;
    double el = (double)e * LN2;
    return el + lm;
}

/* Philox stream layout used for every draw of the method (shared spec, not
 * shared code): key = (seed, stream_id); counter = (index, block, tag, 0). */
enum {
    OR_TAG_DENSE = 0x10,
    OR_TAG_CIRC = 0x11,
    OR_TAG_PERM = 0x12,
    OR_TAG_SIGN = 0x13,
    OR_TAG_CIRC_PM1 = 0x16,
    OR_TAG_TOEP = 0x17,
    OR_TAG_HOUSE = 0x18,
    OR_TAG_SKETCH = 0x19,
    OR_TAG_SKETCH_TOEP = 0x1A
};
#define OR_POLAR_BLOCKS 32

/* One standard normal by Marsaglia's polar method: draw (v1, v2) uniform on
 * [-1,1)^2, keep the pair if 0 < s = v1^2 + v2^2 < 1 and return
 * v1 * sqrt(-2 ln(s) / s).  Each Philox block yields two candidate pairs;
 * rejected pairs move on to the next block (bounded; the chance that 64
 * pairs are all rejected is 0.215^64 < 1e-42, and then 0 is returned). */
OR_EXPORT double or_gauss(uint64_t seed, uint64_t stream, uint64_t tag, uint64_t idx) {
    uint64_t key[2] = {seed, stream};
    for (uint64_t blk = 0; blk < OR_POLAR_BLOCKS; ++blk) {
        uint64_t ctr[4] = {idx, blk, tag, 0}, w[4];
        or_philox4x64_10(ctr, key, w);
        for (int p = 0; p < 2; ++p) {
            double u1 = or_u53(w[2 * p]), u2 = or_u53(w[2 * p + 1]);
            double v1 = 2.0 * u1 - 1.0, v2 = 2.0 * u2 - 1.0;
            double a = v1 * v1, c = v2 * v2;
            double s = a + c;
            if (s > 0.0 && s < 1.0) {
                double t = or_log(s);
                t = -2.0 * t;
                t = t / s;
                t = sqrt(t);
                return v1 * t;
            }
        }
    }
    return 0.0;
}

/* The same polar method carried out in IEEE single precision (used for
 * multipliers on the FP32 grid): 24-bit uniforms, the atanh series to f^11
 * (|f| <= 0.1716 leaves a truncation below 2^-27), single-precision +, -,
 * *, / and sqrt.  Tags are those of the double-precision draws plus 4. */
OR_EXPORT float or_log_f32(float s) {
    uint32_t b;
    memcpy(&b, &s, 4);
    int e = (int)((b >> 23) & 0xff) - 127;
    uint32_t mb = (b & 0x007FFFFFu) | (127u << 23);
    float m;
    memcpy(&m, &mb, 4);
    const float SQRT2F = 1.41421354f, LN2F = 0.693147182f;
    if (m > SQRT2F) { m = m * 0.5f; e = e + 1; }
    float f = (m - 1.0f) / (m + 1.0f);
    float f2 = f * f;
    const int K = 5;
    float p = 1.0f / (float)(2 * K + 1);
    for (int k = K - 1; k >= 0; --k) {
        float t = p * f2;
        p = t + 1.0f / (float)(2 * k + 1);
    }
    float tf = 2.0f * f;
    float lm = tf * p;
    float el = (float)e * LN2F;
    return el + lm;
}

OR_EXPORT float or_gauss_f32(uint64_t seed, uint64_t stream, uint64_t tag, uint64_t idx) {
    uint64_t key[2] = {seed, stream};
    for (uint64_t blk = 0; blk < OR_POLAR_BLOCKS; ++blk) {
        uint64_t ctr[4] = {idx, blk, tag, 0}, w[4];
        or_philox4x64_10(ctr, key, w);
        for (int p = 0; p < 2; ++p) {
            float u1 = (float)(uint32_t)(w[2 * p] >> 40) * 0x1.0p-24f;
            float u2 = (float)(uint32_t)(w[2 * p + 1] >> 40) * 0x1.0p-24f;
            float v1 = 2.0f * u1 - 1.0f, v2 = 2.0f * u2 - 1.0f;
            float a = v1 * v1, c = v2 * v2;
            float s = a + c;
            if (s > 0.0f && s < 1.0f) {
                float t = or_log_f32(s);
                t = -2.0f * t;
                t = t / s;
                t = sqrtf(t);
                return v1 * t;
            }
        }
    }
    return 0.0f;
}

/* Dense Gaussian multiplier drawn in single precision (FP32 grid):
 * G[i][j] = fl32(scale * z32(i*n + j)), scale rounded to float first. */
OR_EXPORT void or_mult_dense_f32(int64_t n, uint64_t seed, uint64_t stream, float scale, double *G, int64_t ldg) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j)
            G[i * ldg + j] = (double)(or_gauss_f32(seed, stream, OR_TAG_DENSE + 4, (uint64_t)(i * n + j)) * scale);
}

OR_EXPORT void or_mult_circulant_f32(int64_t n, uint64_t seed, uint64_t stream, float scale, double *g) {
    for (int64_t i = 0; i < n; ++i)
        g[i] = (double)(or_gauss_f32(seed, stream, OR_TAG_CIRC + 4, (uint64_t)i) * scale);
}

/* Dense Gaussian multiplier (Definition 3.2, G in G_{0,scale}^{n x n}):
 * G[i][j] = scale * z(i*n + j). */
OR_EXPORT void or_mult_dense(int64_t n, uint64_t seed, uint64_t stream, double scale,
                             double *G, int64_t ldg) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j)
            G[i * ldg + j] = or_gauss(seed, stream, OR_TAG_DENSE, (uint64_t)(i * n + j)) * scale;
}

/* Gaussian circulant multiplier (Definition 3.2, Z_{0,scale}): first column
 * g[i] = scale * z(i); the matrix is G[i][j] = g[(i - j) mod n] (Sec. 2.3). */
OR_EXPORT void or_mult_circulant(int64_t n, uint64_t seed, uint64_t stream, double scale,
                                 double *g) {
    for (int64_t i = 0; i < n; ++i) g[i] = or_gauss(seed, stream, OR_TAG_CIRC, (uint64_t)i) * scale;
}

/* Whether the circulant with first column g (entries +-1) is singular at a
 * DFT frequency whose order is a power of two, tested exactly in integers:
 * the bin at frequency 0 vanishes iff sum g_i = 0; the bins at the primitive
 * 2m-th roots of unity w (2m dividing n, m = 1, 2, 4, ...) vanish iff
 * x^m + 1 divides g(x) = sum g_i x^i, i.e. iff every folded sum
 * h_r = sum_q (-1)^q g_{r + q m}, r < m, is zero (g(w) = sum_r h_r w^r and
 * x^m + 1 is irreducible over the rationals).  For n a power of two these are
 * all of the DFT bins (the eigenvalues of the circulant, Sec. 2.3), so the
 * test is exact; for other n it covers the bins of power-of-two order only. */
OR_EXPORT int or_circulant_pm1_singular(int64_t n, const double *g) {
    long long dc = 0;
    for (int64_t i = 0; i < n; ++i) dc += (long long)g[i];
    if (dc == 0) return 1;
    for (int64_t m = 1; 2 * m <= n && n % (2 * m) == 0; m *= 2) {
        int all_zero = 1;
        for (int64_t r = 0; r < m && all_zero; ++r) {
            long long h = 0;
            for (int64_t q = 0; q < n / m; ++q) h += ((q & 1) ? -1 : 1) * (long long)g[r + q * m];
            if (h != 0) all_zero = 0;
        }
        if (all_zero) return 1;
    }
    return 0;
}

/* Circulant multiplier with a first column of random signs (the multipliers
 * of the paper's tests, Sec. 7.1): attempt a draws g_i = +-1 from the low bit
 * of Philox word 0 at counter (i, 0, tag, a); the first attempt whose
 * circulant passes the singularity test above is kept (the paper's remedy
 * for a failure is a fresh draw, Sec. 5).  Returns the attempt used (64 if
 * none of 64 attempts passed: the last one is kept). */
OR_EXPORT int or_mult_circulant_pm1(int64_t n, uint64_t seed, uint64_t stream, double *g) {
    uint64_t key[2] = {seed, stream};
    int a = 0;
    for (; a < 64; ++a) {
        for (int64_t i = 0; i < n; ++i) {
            uint64_t ctr[4] = {(uint64_t)i, 0, OR_TAG_CIRC_PM1, (uint64_t)a}, w[4];
            or_philox4x64_10(ctr, key, w);
            g[i] = (w[0] & 1ull) ? -1.0 : 1.0;
        }
        if (!or_circulant_pm1_singular(n, g)) return a;
    }
    return a;
}

/* Uniform integer in [0, range) from 64-bit words by Lemire's multiply-shift
 * with rejection ("Fast Random Integer Generation in an Interval", ACM TOMACS
 * 2019).  Words come from Philox blocks (i, blk, tag, t). */
static uint64_t or_bounded(uint64_t range, uint64_t seed, uint64_t stream, uint64_t i,
                           uint64_t t) {
    uint64_t key[2] = {seed, stream};
    uint64_t thr = (0 - range) % range;
    uint64_t hi = 0, lo;
    for (uint64_t blk = 0; blk < 16; ++blk) {
        uint64_t ctr[4] = {i, blk, OR_TAG_PERM, t}, w[4];
        or_philox4x64_10(ctr, key, w);
        for (int q = 0; q < 4; ++q) {
            mulhilo64(w[q], range, &hi, &lo);
            if (lo >= thr) return hi;
        }
    }
    return hi;
}

/* Sparse +-1 multiplier G = sum_{t<nnz} D_t P_t: P_t are independent uniform
 * permutations (Fisher-Yates / Durstenfeld: for i = n-1 .. 1 swap p[i] with
 * p[j], j uniform in [0, i]), D_t diagonal random signs.  Column j has its
 * t-th nonzero at row rows[t*n + j] = p_t[j] with value signs[t*n + j].
 * Coinciding rows add up. */
OR_EXPORT void or_mult_sparse(int64_t n, int nnz, uint64_t seed, uint64_t stream, int32_t *rows,
                              int8_t *signs) {
    uint64_t key[2] = {seed, stream};
    for (int t = 0; t < nnz; ++t) {
        int32_t *p = rows + (int64_t)t * n;
        for (int64_t j = 0; j < n; ++j) p[j] = (int32_t)j;
        for (int64_t i = n - 1; i >= 1; --i) {
            int64_t j = (int64_t)or_bounded((uint64_t)(i + 1), seed, stream, (uint64_t)i, (uint64_t)t);
            int32_t tmp = p[i];
            p[i] = p[j];
            p[j] = tmp;
        }
        for (int64_t j = 0; j < n; ++j) {
            uint64_t ctr[4] = {(uint64_t)j, 0, OR_TAG_SIGN, (uint64_t)t}, w[4];
            or_philox4x64_10(ctr, key, w);
            signs[(int64_t)t * n + j] = (w[0] & 1ULL) ? (int8_t)-1 : (int8_t)1;
        }
    }
}

/* Gaussian Toeplitz multiplier (Definition 3.2, T_{0,scale}^{n x n}): only
 * the 2n - 1 entries of the first row and column are independent.  With
 * d = i - j in [-(n-1), n-1], t[d + n - 1] = scale * z(d + n - 1) on its own
 * tag, and T[i][j] = t_{i-j}. */
OR_EXPORT void or_mult_toeplitz(int64_t n, uint64_t seed, uint64_t stream, double scale, double *t) {
    for (int64_t d = 0; d < 2 * n - 1; ++d) t[d] = or_gauss(seed, stream, OR_TAG_TOEP, (uint64_t)d) * scale;
}

OR_EXPORT void or_mult_toeplitz_f32(int64_t n, uint64_t seed, uint64_t stream, float scale, double *t) {
    for (int64_t d = 0; d < 2 * n - 1; ++d)
        t[d] = (double)(or_gauss_f32(seed, stream, OR_TAG_TOEP + 4, (uint64_t)d) * scale);
}

OR_EXPORT void or_toeplitz_to_dense(int64_t n, const double *t, double *G, int64_t ldg) {
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) G[i * ldg + j] = t[i - j + n - 1];
}

/* Householder multiplier with a vector of random signs (the multipliers of
 * the tests the paper cites in Sec. 7.1).  The printed form I - u v^T/(u^T v)
 * is a projection (singular); this is the orthogonal reflector
 * H = I - 2 u u^T / (u^T u) with u^T u = n: u_i = +-1 from the low bit of
 * Philox word 0 at counter (i, 0, tag, 0). */
OR_EXPORT void or_mult_householder_pm1(int64_t n, uint64_t seed, uint64_t stream, double *u) {
    uint64_t key[2] = {seed, stream};
    for (int64_t i = 0; i < n; ++i) {
        uint64_t ctr[4] = {(uint64_t)i, 0, OR_TAG_HOUSE, 0}, w[4];
        or_philox4x64_10(ctr, key, w);
        u[i] = (w[0] & 1ull) ? -1.0 : 1.0;
    }
}

/* H[i][j] = delta_ij - 2 u_i u_j / n. */
OR_EXPORT void or_householder_to_dense(int64_t n, const double *u, double *G, int64_t ldg) {
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
            double v = 2.0 * u[i] * u[j];
            v = v / (double)n;
            G[i * ldg + j] = (i == j ? 1.0 : 0.0) - v;
        }
}

/* Rectangular multipliers of the low-rank approximation (Proto-Alg. 5.1,
 * Stage 1, and the tests of Sec. 7.2), m x r, scale^2 the variance:
 *  Gaussian G[i][j] = scale z(i r + j) on its own tag;
 *  Toeplitz G[i][j] = t_{i-j}, d = i - j in [-(r-1), m-1] drawn at index
 *  d + r - 1 (m + r - 1 independent entries). */
OR_EXPORT void or_mult_sketch(int64_t m, int64_t r, int toeplitz, uint64_t seed, uint64_t stream, double scale,
                              double *G, int64_t ldg) {
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < r; ++j) {
            if (toeplitz) G[i * ldg + j] = or_gauss(seed, stream, OR_TAG_SKETCH_TOEP, (uint64_t)(i - j + r - 1)) * scale;
            else G[i * ldg + j] = or_gauss(seed, stream, OR_TAG_SKETCH, (uint64_t)(i * r + j)) * scale;
        }
}

/* Expand a circulant first column into the full n x n matrix. */
OR_EXPORT void or_circulant_to_dense(int64_t n, const double *g, double *G, int64_t ldg) {
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) G[i * ldg + j] = g[((i - j) % n + n) % n];
}

/* Expand the sparse description into the full n x n matrix. */
OR_EXPORT void or_sparse_to_dense(int64_t n, int nnz, const int32_t *rows, const int8_t *signs,
                                  double *G, int64_t ldg) {
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) G[i * ldg + j] = 0.0;
    for (int t = 0; t < nnz; ++t)
        for (int64_t j = 0; j < n; ++j)
            G[(int64_t)rows[(int64_t)t * n + j] * ldg + j] += (double)signs[(int64_t)t * n + j];
}

/* ------------------------------------------------------------------------ */
/* Dense linear algebra, definitions written out.                            */
/* ------------------------------------------------------------------------ */

/* C = A * B  (m x k times k x n), c_rj = sum_i a_ri b_ij, i ascending. */
OR_EXPORT void or_matmul(int64_t m, int64_t k, int64_t n, const double *A, int64_t lda,
                         const double *B, int64_t ldb, double *C, int64_t ldc) {
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < m; ++r) {
        double *c = C + r * ldc;
        for (int64_t j = 0; j < n; ++j) c[j] = 0.0;
        for (int64_t i = 0; i < k; ++i) {
            double a = A[r * lda + i];
            const double *b = B + i * ldb;
            for (int64_t j = 0; j < n; ++j) c[j] = c[j] + a * b[j];
        }
    }
}

/* Gaussian elimination with no pivoting (Sec. 1.1), unblocked, kji order,
 * in place: on return the strict lower triangle holds L (unit diagonal
 * implied) and the upper triangle holds U, with C = L U.  Returns -1 on
 * success or the first step k whose pivot is zero or not finite (the
 * elimination stops there). */
OR_EXPORT int64_t or_genp(int64_t n, double *C, int64_t ldc) {
    for (int64_t k = 0; k < n; ++k) {
        double p = C[k * ldc + k];
        if (p == 0.0 || !isfinite(p)) return k;
#pragma omp parallel for schedule(static) if (n - k > 256)
        for (int64_t i = k + 1; i < n; ++i) {
            double l = C[i * ldc + k] / p;
            C[i * ldc + k] = l;
            double *ci = C + i * ldc;
            const double *ck = C + k * ldc;
            for (int64_t j = k + 1; j < n; ++j) ci[j] = ci[j] - l * ck[j];
        }
    }
    return -1;
}

/* Gaussian elimination with partial pivoting: at step k the pivot row is the
 * first i >= k with the largest |a_ik| (the LAPACK idamax convention); rows
 * k and piv[k] are swapped across the whole matrix.  Same kji update order
 * as or_genp, so on inputs that need no swap the two agree bit for bit.
 * Returns -1 or the first step with an all-zero pivot column. */
OR_EXPORT int64_t or_gepp(int64_t n, double *A, int64_t lda, int64_t *piv) {
    for (int64_t k = 0; k < n; ++k) {
        int64_t pr = k;
        double best = fabs(A[k * lda + k]);
        for (int64_t i = k + 1; i < n; ++i) {
            double v = fabs(A[i * lda + k]);
            if (v > best) { best = v; pr = i; }
        }
        piv[k] = pr;
        if (best == 0.0 || !isfinite(best)) return k;
        if (pr != k)
            for (int64_t j = 0; j < n; ++j) {
                double t = A[k * lda + j];
                A[k * lda + j] = A[pr * lda + j];
                A[pr * lda + j] = t;
            }
        double p = A[k * lda + k];
#pragma omp parallel for schedule(static) if (n - k > 256)
        for (int64_t i = k + 1; i < n; ++i) {
            double l = A[i * lda + k] / p;
            A[i * lda + k] = l;
            double *ai = A + i * lda;
            const double *ak = A + k * lda;
            for (int64_t j = k + 1; j < n; ++j) ai[j] = ai[j] - l * ak[j];
        }
    }
    return -1;
}

/* Forward substitution with the unit lower factor stored below the diagonal
 * of LU: B <- L^{-1} B, B is n x nrhs. */
OR_EXPORT void or_solve_lower_unit(int64_t n, int64_t nrhs, const double *LU, int64_t ld,
                                   double *B, int64_t ldb) {
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = 0; k < i; ++k) {
            double l = LU[i * ld + k];
            for (int64_t c = 0; c < nrhs; ++c) B[i * ldb + c] = B[i * ldb + c] - l * B[k * ldb + c];
        }
}

/* Back substitution with the upper factor: B <- U^{-1} B. */
OR_EXPORT void or_solve_upper(int64_t n, int64_t nrhs, const double *LU, int64_t ld, double *B,
                              int64_t ldb) {
    for (int64_t i = n - 1; i >= 0; --i) {
        for (int64_t k = i + 1; k < n; ++k) {
            double u = LU[i * ld + k];
            for (int64_t c = 0; c < nrhs; ++c) B[i * ldb + c] = B[i * ldb + c] - u * B[k * ldb + c];
        }
        double d = LU[i * ld + i];
        for (int64_t c = 0; c < nrhs; ++c) B[i * ldb + c] = B[i * ldb + c] / d;
    }
}

/* Transposed solves for the adjoint: B <- U^{-T} B, then B <- L^{-T} B. */
OR_EXPORT void or_solve_upper_T(int64_t n, int64_t nrhs, const double *LU, int64_t ld, double *B,
                                int64_t ldb) {
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t k = 0; k < i; ++k) {
            double u = LU[k * ld + i];
            for (int64_t c = 0; c < nrhs; ++c) B[i * ldb + c] = B[i * ldb + c] - u * B[k * ldb + c];
        }
        double d = LU[i * ld + i];
        for (int64_t c = 0; c < nrhs; ++c) B[i * ldb + c] = B[i * ldb + c] / d;
    }
}

OR_EXPORT void or_solve_lower_unit_T(int64_t n, int64_t nrhs, const double *LU, int64_t ld,
                                     double *B, int64_t ldb) {
    for (int64_t i = n - 1; i >= 0; --i)
        for (int64_t k = i + 1; k < n; ++k) {
            double l = LU[k * ld + i];
            for (int64_t c = 0; c < nrhs; ++c) B[i * ldb + c] = B[i * ldb + c] - l * B[k * ldb + c];
        }
}

/* Apply the row swaps recorded by or_gepp to B (P B). */
OR_EXPORT void or_apply_piv(int64_t n, int64_t nrhs, const int64_t *piv, double *B, int64_t ldb) {
    for (int64_t k = 0; k < n; ++k)
        if (piv[k] != k)
            for (int64_t c = 0; c < nrhs; ++c) {
                double t = B[k * ldb + c];
                B[k * ldb + c] = B[piv[k] * ldb + c];
                B[piv[k] * ldb + c] = t;
            }
}

/* Undo the row permutation of GEPP for a transposed solve: B <- P^T B. */
OR_EXPORT void or_apply_piv_T(int64_t n, int64_t nrhs, const int64_t *piv, double *B, int64_t ldb) {
    for (int64_t k = n - 1; k >= 0; --k)
        if (piv[k] != k)
            for (int64_t c = 0; c < nrhs; ++c) {
                double t = B[k * ldb + c];
                B[k * ldb + c] = B[piv[k] * ldb + c];
                B[piv[k] * ldb + c] = t;
            }
}

/* R = B - A X  (A n x n, X and B n x nrhs). */
OR_EXPORT void or_residual(int64_t n, int64_t nrhs, const double *A, int64_t lda, const double *X,
                           int64_t ldx, const double *B, int64_t ldb, double *R, int64_t ldr) {
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n; ++r) {
        for (int64_t c = 0; c < nrhs; ++c) {
            double s = 0.0;
            for (int64_t j = 0; j < n; ++j) s = s + A[r * lda + j] * X[j * ldx + c];
            R[r * ldr + c] = B[r * ldb + c] - s;
        }
    }
}

/* Normwise backward error of each column (Rigal & Gaches):
 * eta_c = ||b_c - A x_c||_inf / (||A||_inf ||x_c||_inf + ||b_c||_inf);
 * the maximum over columns is returned. */
OR_EXPORT double or_backward_error(int64_t n, int64_t nrhs, const double *A, int64_t lda,
                                   const double *X, int64_t ldx, const double *B, int64_t ldb) {
    double anorm = 0.0;
    for (int64_t r = 0; r < n; ++r) {
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) s = s + fabs(A[r * lda + j]);
        if (s > anorm) anorm = s;
    }
    double *R = (double *)malloc((size_t)(n * nrhs) * sizeof(double));
    or_residual(n, nrhs, A, lda, X, ldx, B, ldb, R, nrhs);
    double worst = 0.0;
    for (int64_t c = 0; c < nrhs; ++c) {
        double rn = 0.0, xn = 0.0, bn = 0.0;
        for (int64_t r = 0; r < n; ++r) {
            if (fabs(R[r * nrhs + c]) > rn) rn = fabs(R[r * nrhs + c]);
            if (fabs(X[r * ldx + c]) > xn) xn = fabs(X[r * ldx + c]);
            if (fabs(B[r * ldb + c]) > bn) bn = fabs(B[r * ldb + c]);
        }
        double eta = rn / (anorm * xn + bn);
        if (eta > worst) worst = eta;
    }
    free(R);
    return worst;
}

/* ------------------------------------------------------------------------ */
/* Products with the structured multipliers, from their definitions.         */
/* ------------------------------------------------------------------------ */

/* C = A * G for circulant G[i][j] = g[(i-j) mod n], m rows of A:
 * c_rj = sum_i a_ri g[(i-j) mod n]. */
OR_EXPORT void or_circ_matmul(int64_t m, int64_t n, const double *A, int64_t lda, const double *g,
                              double *C, int64_t ldc) {
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < m; ++r)
        for (int64_t j = 0; j < n; ++j) {
            double s = 0.0;
            for (int64_t i = 0; i < n; ++i) s = s + A[r * lda + i] * g[((i - j) % n + n) % n];
            C[r * ldc + j] = s;
        }
}

/* C = A * G for the sparse G: c_rj = sum_t s_tj a_{r, rows_tj}, t ascending. */
OR_EXPORT void or_sparse_matmul(int64_t m, int64_t n, int nnz, const double *A, int64_t lda,
                                const int32_t *rows, const int8_t *signs, double *C, int64_t ldc) {
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < m; ++r)
        for (int64_t j = 0; j < n; ++j) {
            double s = 0.0;
            for (int t = 0; t < nnz; ++t)
                s = s + (double)signs[(int64_t)t * n + j] * A[r * lda + rows[(int64_t)t * n + j]];
            C[r * ldc + j] = s;
        }
}

/* X = G * Y (trans = 0) or X = G^T * Y (trans = 1) for circulant G,
 * Y and X n x nrhs: x_i = sum_j G[i][j] y_j. */
OR_EXPORT void or_circ_apply(int64_t n, int64_t nrhs, int trans, const double *g, const double *Y,
                             int64_t ldy, double *X, int64_t ldx) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t c = 0; c < nrhs; ++c) {
            double s = 0.0;
            for (int64_t j = 0; j < n; ++j) {
                int64_t d = trans ? (j - i) : (i - j);
                s = s + g[(d % n + n) % n] * Y[j * ldy + c];
            }
            X[i * ldx + c] = s;
        }
}

/* X = G * Y or G^T * Y for the sparse G. */
OR_EXPORT void or_sparse_apply(int64_t n, int64_t nrhs, int trans, int nnz, const int32_t *rows,
                               const int8_t *signs, const double *Y, int64_t ldy, double *X,
                               int64_t ldx) {
    for (int64_t i = 0; i < n; ++i)
        for (int64_t c = 0; c < nrhs; ++c) X[i * ldx + c] = 0.0;
    for (int t = 0; t < nnz; ++t)
        for (int64_t j = 0; j < n; ++j) {
            int64_t r = rows[(int64_t)t * n + j];
            double s = (double)signs[(int64_t)t * n + j];
            for (int64_t c = 0; c < nrhs; ++c) {
                if (trans) X[j * ldx + c] = X[j * ldx + c] + s * Y[r * ldy + c];
                else X[r * ldx + c] = X[r * ldx + c] + s * Y[j * ldy + c];
            }
        }
}

/* ------------------------------------------------------------------------ */
/* Block Gaussian elimination with explicit inverses of the pivot blocks     */
/* (Sec. 2: Theorem 2.2 bounds the norms of the pivot blocks of block        */
/* Gaussian elimination and of their inverses for a strongly well            */
/* conditioned matrix).  C is cut into diagonal blocks of order nb (the last */
/* one ragged).  At step k the leading block of the current Schur complement */
/* is the pivot block P_k; it is inverted explicitly, the block column below */
/* it becomes L_ik = S_ik P_k^{-1}, the block row stays (U_kj = S_kj), and   */
/* the rest is updated, S_ij <- S_ij - L_ik S_kj.  So C = L_B U_B with L_B   */
/* block unit lower (identity diagonal blocks) and U_B block upper with the  */
/* pivot blocks on its diagonal.                                             */
/* ------------------------------------------------------------------------ */

/* X = P^{-1} for the kb x kb block P (ld ldp) by Gauss-Jordan elimination
 * without pivoting on [P | I]: at step t divide row t by its pivot, then
 * clear column t from every other row.  X is written with leading dimension
 * ldx.  Returns -1, or the first step t whose pivot is zero or not finite
 * (P's leading t+1 minor is singular, or the arithmetic overflowed). */
OR_EXPORT int64_t or_gauss_jordan_inverse(int64_t kb, const double *P, int64_t ldp, double *X, int64_t ldx) {
    double *M = (double *)malloc((size_t)(kb * kb > 0 ? kb * kb : 1) * sizeof(double));
    if (!M) return -2;
    for (int64_t i = 0; i < kb; ++i)
        for (int64_t j = 0; j < kb; ++j) {
            M[i * kb + j] = P[i * ldp + j];
            X[i * ldx + j] = (i == j) ? 1.0 : 0.0;
        }
    for (int64_t t = 0; t < kb; ++t) {
        double p = M[t * kb + t];
        if (p == 0.0 || !isfinite(p)) {
            free(M);
            return t;
        }
        for (int64_t j = 0; j < kb; ++j) {
            M[t * kb + j] = M[t * kb + j] / p;
            X[t * ldx + j] = X[t * ldx + j] / p;
        }
        for (int64_t i = 0; i < kb; ++i) {
            if (i == t) continue;
            double f = M[i * kb + t];
            for (int64_t j = 0; j < kb; ++j) {
                M[i * kb + j] = M[i * kb + j] - f * M[t * kb + j];
                X[i * ldx + j] = X[i * ldx + j] - f * X[t * ldx + j];
            }
        }
    }
    free(M);
    return -1;
}

/* Block GE of C in place.  On return the blocks strictly below the block
 * diagonal hold L_B, the blocks on and above it hold U_B (the pivot blocks
 * P_k themselves on the diagonal), and Pinv[k nb nb + r nb + c] holds
 * (P_k^{-1})[r][c] (a ragged last block of order kb uses its top-left
 * kb x kb).  Returns -1, or the global index k0 + t of the first zero /
 * non-finite pivot met while inverting P_k. */
OR_EXPORT int64_t or_block_genp(int64_t n, double *C, int64_t ldc, int64_t nb, double *Pinv) {
    double *row = (double *)malloc((size_t)(nb > 0 ? nb : 1) * sizeof(double));
    if (!row) return -2;
    for (int64_t k0 = 0; k0 < n; k0 += nb) {
        const int64_t kb = (n - k0 < nb) ? n - k0 : nb;
        double *X = Pinv + (k0 / nb) * nb * nb;
        int64_t t = or_gauss_jordan_inverse(kb, C + k0 * ldc + k0, ldc, X, nb);
        if (t >= 0) {
            free(row);
            return t == -2 ? -2 : k0 + t;
        }
        const int64_t e0 = k0 + kb;
        /* L_ik = S_ik P_k^{-1}, one row at a time */
        for (int64_t i = e0; i < n; ++i) {
            double *ci = C + i * ldc + k0;
            for (int64_t c = 0; c < kb; ++c) {
                double s = 0.0;
                for (int64_t r = 0; r < kb; ++r) s = s + ci[r] * X[r * nb + c];
                row[c] = s;
            }
            for (int64_t c = 0; c < kb; ++c) ci[c] = row[c];
        }
        /* S_ij <- S_ij - L_ik S_kj */
#pragma omp parallel for schedule(static) if (n - e0 > 256)
        for (int64_t i = e0; i < n; ++i) {
            double *ci = C + i * ldc;
            for (int64_t r = 0; r < kb; ++r) {
                const double l = ci[k0 + r];
                const double *ur = C + (k0 + r) * ldc;
                for (int64_t j = e0; j < n; ++j) ci[j] = ci[j] - l * ur[j];
            }
        }
    }
    free(row);
    return -1;
}

/* Y <- U_B^{-1} L_B^{-1} Y for block GE factors: block forward substitution
 * with L_B (z_i = b_i - sum_{k<i} L_ik z_k), then block back substitution
 * with U_B (y_i = P_i^{-1} (z_i - sum_{j>i} U_ij y_j)). */
OR_EXPORT void or_block_lu_solve(int64_t n, int64_t nrhs, const double *LU, int64_t ld, int64_t nb,
                                 const double *Pinv, double *Y, int64_t ldy) {
    double *tmp = (double *)malloc((size_t)(nb > 0 ? nb : 1) * sizeof(double));
    if (!tmp) return;
    for (int64_t c = 0; c < nrhs; ++c) {
        for (int64_t i0 = 0; i0 < n; i0 += nb) {
            const int64_t ib = (n - i0 < nb) ? n - i0 : nb;
            for (int64_t r = 0; r < ib; ++r) {
                double s = Y[(i0 + r) * ldy + c];
                for (int64_t k = 0; k < i0; ++k) s = s - LU[(i0 + r) * ld + k] * Y[k * ldy + c];
                Y[(i0 + r) * ldy + c] = s;
            }
        }
        int64_t last = ((n - 1) / nb) * nb;
        for (int64_t i0 = last; i0 >= 0; i0 -= nb) {
            const int64_t ib = (n - i0 < nb) ? n - i0 : nb;
            const double *X = Pinv + (i0 / nb) * nb * nb;
            for (int64_t r = 0; r < ib; ++r) {
                double s = Y[(i0 + r) * ldy + c];
                for (int64_t j = i0 + ib; j < n; ++j) s = s - LU[(i0 + r) * ld + j] * Y[j * ldy + c];
                tmp[r] = s;
            }
            for (int64_t r = 0; r < ib; ++r) {
                double s = 0.0;
                for (int64_t q = 0; q < ib; ++q) s = s + X[r * nb + q] * tmp[q];
                Y[(i0 + r) * ldy + c] = s;
            }
        }
    }
    free(tmp);
}
