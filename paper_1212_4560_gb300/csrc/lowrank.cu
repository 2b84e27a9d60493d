// lowrank.cu -- randomized low-rank approximation (Sec. 5, Proto-Alg. 5.1,
// with an orthonormal T as in the tests of Sec. 7.2):
//   Stage 1   B = A^T G,   G an m x r Gaussian (Definition 3.2) or Gaussian
//             Toeplitz sketch (Table 7.3);
//   basis     B = Q R with R upper triangular, positive diagonal (Q is then
//             unique, Fact 2.2), by shifted Cholesky QR: R1^T R1 = B^T B + s I,
//             Q1 = B R1^{-1}, then two unshifted passes (CholeskyQR3:
//             Fukaya, Kannan, Nakatsukasa, Yamamoto & Yanagisawa, SIAM J.
//             Sci. Comput. 2020), which stays orthogonal for kappa(B) up to
//             about 1/u; R = Q^T B;
//   Stage 3   A Q, so A_hat = A T (T^T T)^{-1} T^T = (A Q) Q^T.
// Everything but the r x r Cholesky factorizations runs in the FP64 GEMM
// kernels (B^T B, A^T G, A Q) and a row-parallel triangular solve.
// Also the numerical rank of App. B (Proto-Alg. B.1): the largest r whose
// sketch A^T G_r is well conditioned, by binary search, its COND test by
// power and inverse iteration on the sketch's Gram matrix (Remark B.2).
#include "genp_internal.cuh"

#include <math.h>

namespace genp {
namespace {

constexpr int kMaxR = 128;   // r x r Gram matrix in shared memory

// Cholesky S + shift I = R^T R (upper R, r <= kMaxR) in one CTA, in place in
// shared memory; R written to Rout (ld r).  shift_mult > 0: the shift is
// shift_mult * trace(S) (CholeskyQR3's first pass: 11 (n r + r (r + 1)) u
// ||B||_F^2).  A non-positive or non-finite pivot at step k sets *fail = k + 1.
__global__ void __launch_bounds__(256) k_chol(const double *S, int r, double shift_mult, double *Rout, int *fail) {
    extern __shared__ double a[];   // r x r, ld r + 1
    const int ld = r + 1, tid = threadIdx.x;
    for (int idx = tid; idx < r * r; idx += blockDim.x) a[(idx / r) * ld + idx % r] = S[idx];
    __syncthreads();
    __shared__ double sh;
    if (tid == 0) {
        double tr = 0.0;
        for (int i = 0; i < r; ++i) tr += a[i * ld + i];
        sh = shift_mult * tr;
    }
    __syncthreads();
    for (int i = tid; i < r; i += blockDim.x) a[i * ld + i] += sh;
    __syncthreads();
    __shared__ int bad;
    if (tid == 0) bad = 0;
    __syncthreads();
    for (int k = 0; k < r; ++k) {
        if (tid == 0) {
            const double d = a[k * ld + k];
            if (!(d > 0.0) || !isfinite(d)) {
                if (!bad) bad = k + 1;
                a[k * ld + k] = 1.0;
            } else {
                a[k * ld + k] = sqrt(d);
            }
        }
        __syncthreads();
        const double p = a[k * ld + k];
        for (int j = k + 1 + tid; j < r; j += blockDim.x) a[k * ld + j] /= p;   // row k of R
        __syncthreads();
        const int rem = r - k - 1;
        for (int idx = tid; idx < rem * rem; idx += blockDim.x) {
            const int i = k + 1 + idx / rem, j = k + 1 + idx % rem;
            if (j >= i) a[i * ld + j] = fma(-a[k * ld + i], a[k * ld + j], a[i * ld + j]);
        }
        __syncthreads();
    }
    for (int idx = tid; idx < r * r; idx += blockDim.x) {
        const int i = idx / r, j = idx % r;
        Rout[idx] = j >= i ? a[i * ld + j] : 0.0;
    }
    if (tid == 0 && bad && fail) atomicCAS(fail, 0, bad);
}

// X = Y R^{-1} row by row (R upper, r x r), one thread per row of Y.
__global__ void __launch_bounds__(128) k_right_solve_upper(const double *Y, int64_t ldy, int64_t nrows, int r,
                                                           const double *R, double *X, int64_t ldx) {
    extern __shared__ double rs[];   // R, ld r
    for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) rs[idx] = R[idx];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nrows; i += (int64_t)gridDim.x * blockDim.x) {
        const double *y = Y + i * ldy;
        double *x = X + i * ldx;
        for (int j = 0; j < r; ++j) {
            double v = y[j];
            for (int k = 0; k < j; ++k) v = fma(-x[k], rs[k * r + j], v);
            x[j] = v / rs[j * r + j];
        }
    }
}

// COND of App. B (Remark B.2: no pivoting, no orthogonalization) for the
// r x r Gram matrix S = B'^T B' of a sketch: Cholesky S = R^T R without
// pivoting (a non-positive pivot: not of full rank), then 40 power steps
// (S v = R^T (R v)) for lambda_max and 40 inverse-iteration steps (solves
// with R^T and R) for lambda_min; out[0] = sqrt(lambda_max / lambda_min) =
// kappa_2(B'), or infinity.  One warp, r <= kMaxR.
__global__ void __launch_bounds__(32) k_cond(const double *S, int r, double *out) {
    extern __shared__ double sm[];
    double *R = sm;                 // Cholesky factor, ld r + 1
    double *v = R + r * (r + 1);
    double *w = v + r;
    double *u = w + r;
    const int ld = r + 1, lane = threadIdx.x;
    for (int idx = lane; idx < r * r; idx += 32) R[(idx / r) * ld + idx % r] = S[idx];
    __syncwarp();
    bool bad = false;
    for (int k = 0; k < r; ++k) {
        const double d = R[k * ld + k];
        bad = !(d > 0.0) || !isfinite(d);
        if (bad) break;
        const double p = sqrt(d);
        __syncwarp();
        if (lane == 0) R[k * ld + k] = p;
        for (int j = k + 1 + lane; j < r; j += 32) R[k * ld + j] /= p;
        __syncwarp();
        for (int i = k + 1; i < r; ++i)
            for (int j = i + lane; j < r; j += 32) R[i * ld + j] = fma(-R[k * ld + i], R[k * ld + j], R[i * ld + j]);
        __syncwarp();
    }
    if (bad) {
        if (lane == 0) out[0] = INFINITY;
        return;
    }
    auto norm2 = [&](const double *x) {
        double t = 0.0;
        for (int i = lane; i < r; i += 32) t = fma(x[i], x[i], t);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        return sqrt(t);
    };
    // lambda_max: power steps, S v = R^T (R v)
    for (int i = lane; i < r; i += 32) v[i] = 1.0 + 1e-3 * i;
    __syncwarp();
    double lmax = 0.0;
    for (int it = 0; it < 40; ++it) {
        const double nv = norm2(v);
        for (int i = lane; i < r; i += 32) {          // u = R v / ||v||
            double t = 0.0;
            for (int j = i; j < r; ++j) t = fma(R[i * ld + j], v[j], t);
            u[i] = t / nv;
        }
        __syncwarp();
        for (int i = lane; i < r; i += 32) {          // w = R^T u
            double t = 0.0;
            for (int k = 0; k <= i; ++k) t = fma(R[k * ld + i], u[k], t);
            w[i] = t;
        }
        __syncwarp();
        lmax = norm2(w);
        for (int i = lane; i < r; i += 32) v[i] = w[i];
        __syncwarp();
    }
    // lambda_min: inverse iteration, S^{-1} v = R^{-1} R^{-T} v
    for (int i = lane; i < r; i += 32) v[i] = 1.0 + 1e-3 * i;
    __syncwarp();
    double mu = 0.0;
    for (int it = 0; it < 40; ++it) {
        const double nv = norm2(v);
        for (int i = 0; i < r; ++i) {           // R^T y = v / ||v||   (y in w)
            double t = 0.0;
            for (int k = lane; k < i; k += 32) t = fma(R[k * ld + i], w[k], t);
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) w[i] = (v[i] / nv - t) / R[i * ld + i];
            __syncwarp();
        }
        for (int i = r - 1; i >= 0; --i) {      // R z = y   (z in v)
            double t = 0.0;
            for (int k = i + 1 + lane; k < r; k += 32) t = fma(R[i * ld + k], v[k], t);
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) v[i] = (w[i] - t) / R[i * ld + i];
            __syncwarp();
        }
        mu = norm2(v);                          // ~ 1 / lambda_min
    }
    if (lane == 0) {
        const double k2 = lmax * mu;
        out[0] = (k2 > 0.0 && isfinite(k2)) ? sqrt(k2) : INFINITY;
    }
}

}  // namespace

cudaError_t numerical_rank_run(int64_t m, int64_t n, const double *A, int64_t lda, int64_t r_lo, int64_t r_hi,
                               double cond_max, uint64_t seed, uint64_t sid, int64_t *rank, double *B, int64_t ldb,
                               void *work, double *host_kappa, cudaStream_t s) {
    // work: G (m x r_hi), Bp (n x r_hi), S (r_hi x r_hi), kappa (1)
    double *G = static_cast<double *>(work);
    double *Bp = G + m * r_hi;
    double *S = Bp + n * r_hi;
    double *dk = S + r_hi * r_hi;
    cudaError_t e = launch_sketch(G, r_hi, m, r_hi, false, seed, sid, 1.0, s);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_cond, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((kMaxR * (kMaxR + 1) + 3 * kMaxR) * sizeof(double)));
        attr = true;
    }
    int64_t lo = r_lo, hi = r_hi;
    while (lo < hi && e == cudaSuccess) {
        const int64_t r = (lo + hi + 1) / 2;
        e = gemm<double>(n, r, m, 1.0, A, lda, true, G, r_hi, 0.0, nullptr, 0, Bp, r, nullptr, s);   // A^T G_r
        if (e == cudaSuccess) e = gemm<double>(r, r, n, 1.0, Bp, r, true, Bp, r, 0.0, nullptr, 0, S, r, nullptr, s);
        if (e != cudaSuccess) break;
        note_launch();
        k_cond<<<1, 32, (size_t)(r * (r + 1) + 3 * r) * sizeof(double), s>>>(S, (int)r, dk);
        e = cudaMemcpyAsync(host_kappa, dk, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        const double kappa = *host_kappa;
        if (isfinite(kappa) && kappa <= cond_max) lo = r;
        else hi = r - 1;
    }
    if (e == cudaSuccess && B && lo > 0)
        e = gemm<double>(n, lo, m, 1.0, A, lda, true, G, r_hi, 0.0, nullptr, 0, B, ldb, nullptr, s);
    *rank = lo;
    return e;
}

size_t numerical_rank_work_bytes(int64_t m, int64_t n, int64_t r_hi) {
    return (size_t)(m * r_hi + n * r_hi + r_hi * r_hi + 1) * sizeof(double);
}

cudaError_t lowrank_run(int64_t m, int64_t n, const double *A, int64_t lda, int64_t r, bool toeplitz, uint64_t seed,
                        uint64_t sid, double *G, int64_t ldg, double *Q, int64_t ldq, double *R, int64_t ldr,
                        double *AQ, int64_t ldaq, int *fail, void *work, cudaStream_t s) {
    // work: B (n x r), S (r x r), Rk (r x r), T (n x r), G (m x r) if the caller gives none
    double *B = static_cast<double *>(work);
    double *S = B + n * r;
    double *Rk = S + r * r;
    double *T = Rk + r * r;
    if (!G) {
        G = T + n * r;
        ldg = r;
    }
    cudaError_t e = launch_sketch(G, ldg, m, r, toeplitz, seed, sid, 1.0, s);
    if (e == cudaSuccess) e = gemm<double>(n, r, m, 1.0, A, lda, true, G, ldg, 0.0, nullptr, 0, B, r, nullptr, s);
    const double u = 1.1102230246251565e-16;
    const size_t sm_chol = (size_t)r * (r + 1) * sizeof(double), sm_solve = (size_t)r * r * sizeof(double);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kMaxR * (kMaxR + 1) * 8));
        cudaFuncSetAttribute(k_right_solve_upper, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kMaxR * kMaxR * 8));
        attr = true;
    }
    const unsigned rows = (unsigned)cdiv(n, 128) < 152 * 4 ? (unsigned)cdiv(n, 128) : 152 * 4;
    // B -> Q -> T -> Q: each pass factors the Gram matrix of its source and
    // divides the source by that Cholesky factor from the right
    const double *srcs[3] = {B, Q, T};
    const int64_t lds[3] = {r, ldq, r};
    double *dsts[3] = {Q, T, Q};
    const int64_t ldds[3] = {ldq, r, ldq};
    for (int pass = 0; pass < 3 && e == cudaSuccess; ++pass) {
        e = gemm<double>(r, r, n, 1.0, srcs[pass], lds[pass], true, srcs[pass], lds[pass], 0.0, nullptr, 0, S, r,
                         nullptr, s);
        if (e != cudaSuccess) break;
        const double shift = pass == 0 ? 11.0 * ((double)n * r + (double)r * (r + 1)) * u : 0.0;
        note_launch();
        k_chol<<<1, 256, sm_chol, s>>>(S, (int)r, shift, Rk, fail);
        note_launch();
        k_right_solve_upper<<<rows, 128, sm_solve, s>>>(srcs[pass], lds[pass], n, (int)r, Rk, dsts[pass],
                                                        ldds[pass]);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && R) e = gemm<double>(r, r, n, 1.0, Q, ldq, true, B, r, 0.0, nullptr, 0, R, ldr, nullptr, s);
    if (e == cudaSuccess && AQ) e = gemm<double>(m, r, n, 1.0, A, lda, false, Q, ldq, 0.0, nullptr, 0, AQ, ldaq, nullptr, s);
    return e;
}

size_t lowrank_work_bytes(int64_t m, int64_t n, int64_t r) {
    return (size_t)(2 * n * r + 2 * r * r + m * r) * sizeof(double);
}

}  // namespace genp
