// gemm.cu -- register-tiled CUDA-core GEMM, D = alpha * op(A) * B + beta * Cin.
//
// FP64 on GB300 runs at 4 flop/clk/SM on the CUDA cores (2 DFMA/clk/SM;
// mma.sync .f64 measured slower) and there is no FP64 tcgen05 kind, so the
// FP64 contractions of the method (the product A*G of Thm. 4.1 and the
// Schur-complement update of block Gaussian elimination) are DFMA-bound:
// one 64x64 tile per CTA, 4x4 outputs per thread, operand tiles staged in
// shared memory with a register prefetch of the next K slice.  FP32 uses a
// 128x128 tile with 8x8 outputs per thread (FFMA).  The A and B loaders can
// also synthesise a circulant operand G[i][j] = g[(i-j) mod n] on the fly.
#include "genp_internal.cuh"
#include "dfloat.cuh"

namespace genp {

enum Src { kDense = 0, kCirc = 1, kCircT = 2 };

// Matrix-vector launches that found their skip flag set (the device-steered
// refinement enqueues steps it may not need): the launch profile counts the
// work of the others only.
__device__ unsigned int g_gemv_skipped;
__device__ __forceinline__ bool gemv_skipped(const int *skip) {
    if (!(skip && *skip)) return false;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&g_gemv_skipped, 1u);
    return true;
}

template <typename T, int BM, int BN, int BK, int TM, int TN, bool TRANSA, int ASRC, int BSRC>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_gemm(int64_t m, int64_t n, int64_t k, T alpha, const T *__restrict__ A, int64_t lda,
       const T *__restrict__ B, int64_t ldb, T beta, const T *Cin, int64_t ldci, T *D, int64_t ldd,
       const int *skip, const double *g, int64_t gn) {
    if (skip && *skip) return;
    constexpr int NT = (BM / TM) * (BN / TN);
    constexpr int AE = BM * BK / NT, BE = BK * BN / NT;
    static_assert(AE * NT == BM * BK && BE * NT == BK * BN, "tile split");
    __shared__ __align__(16) T As[2][BK][BM];
    __shared__ __align__(16) T Bs[2][BK][BN];
    const int tid = threadIdx.x;
    const int tx = tid % (BN / TN), ty = tid / (BN / TN);
    const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;

    T ra[AE], rb[BE];
    auto circ = [&](int64_t d) -> T {
        d %= gn;
        if (d < 0) d += gn;
        return (T)g[d];
    };
    auto load = [&](int64_t k0) {
#pragma unroll
        for (int e = 0; e < AE; ++e) {
            const int lin = tid + e * NT;
            int r, kk;
            if (!TRANSA) { r = lin / BK; kk = lin % BK; }
            else { kk = lin / BM; r = lin % BM; }
            const int64_t gr = m0 + r, gk = k0 + kk;
            T v = T(0);
            if (gr < m && gk < k) {
                if (ASRC == kDense) v = TRANSA ? A[gk * lda + gr] : A[gr * lda + gk];
                else if (ASRC == kCirc) v = circ(gr - gk);
                else v = circ(gk - gr);
            }
            ra[e] = v;
        }
#pragma unroll
        for (int e = 0; e < BE; ++e) {
            const int lin = tid + e * NT;
            const int kk = lin / BN, c = lin % BN;
            const int64_t gk = k0 + kk, gc = n0 + c;
            T v = T(0);
            if (gk < k && gc < n) v = (BSRC == kDense) ? B[gk * ldb + gc] : circ(gk - gc);
            rb[e] = v;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int e = 0; e < AE; ++e) {
            const int lin = tid + e * NT;
            int r, kk;
            if (!TRANSA) { r = lin / BK; kk = lin % BK; }
            else { kk = lin / BM; r = lin % BM; }
            As[buf][kk][r] = ra[e];
        }
#pragma unroll
        for (int e = 0; e < BE; ++e) {
            const int lin = tid + e * NT;
            Bs[buf][lin / BN][lin % BN] = rb[e];
        }
    };

    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

    const int64_t nkt = (k + BK - 1) / BK;
    load(0);
    store(0);
    __syncthreads();
    for (int64_t kt = 0; kt < nkt; ++kt) {
        const int buf = (int)(kt & 1);
        if (kt + 1 < nkt) load((kt + 1) * BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty * TM + i];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][tx * TN + j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        if (kt + 1 < nkt) store(buf ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t r = m0 + ty * TM + i;
        if (r >= m) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int64_t c = n0 + tx * TN + j;
            if (c >= n) continue;
            T v = alpha * acc[i][j];
            if (beta != T(0)) v = fma(beta, Cin[r * ldci + c], v);
            D[r * ldd + c] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// Skinny products (n <= 16 columns: the right-hand sides of the solves, the
// residual b - A x, x = G y): matrix-vector kernels that read A once,
// coalesced, and compute only the n real columns.
//  op(A) = A:   one warp per RW rows, lanes stride over k, warp-shuffle sums.
//  op(A) = A^T: one lane per output row (a column of A), the CTA's 8 warps
//               split k and add their partial sums in shared memory.
// Both sum in a fixed order (deterministic).
// ---------------------------------------------------------------------------
template <typename T, int NR, int RW>
__global__ void __launch_bounds__(256) k_gemv_n(int64_t m, int nr, int64_t k, T alpha, const T *__restrict__ A,
                                                 int64_t lda, const T *__restrict__ B, int64_t ldb, T beta,
                                                 const T *Cin, int64_t ldci, T *D, int64_t ldd, const int *skip) {
    if (gemv_skipped(skip)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t i0 = ((int64_t)blockIdx.x * 8 + warp) * RW; i0 < m; i0 += (int64_t)gridDim.x * 8 * RW) {
        T acc[RW][NR];
#pragma unroll
        for (int r = 0; r < RW; ++r)
#pragma unroll
            for (int c = 0; c < NR; ++c) acc[r][c] = T(0);
        const T *arow[RW];
#pragma unroll
        for (int r = 0; r < RW; ++r) arow[r] = A + (i0 + r < m ? i0 + r : i0) * lda;
#pragma unroll 8
        for (int64_t kk = lane; kk < k; kk += 32) {
            T b[NR];
#pragma unroll
            for (int c = 0; c < NR; ++c) b[c] = c < nr ? __ldg(B + kk * ldb + c) : T(0);
#pragma unroll
            for (int r = 0; r < RW; ++r) {
                const T a = __ldg(arow[r] + kk);
#pragma unroll
                for (int c = 0; c < NR; ++c) acc[r][c] = fma(a, b[c], acc[r][c]);
            }
        }
#pragma unroll
        for (int r = 0; r < RW; ++r)
#pragma unroll
            for (int c = 0; c < NR; ++c)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc[r][c] += __shfl_xor_sync(0xffffffffu, acc[r][c], o);
        if (lane < NR) {
#pragma unroll
            for (int r = 0; r < RW; ++r) {
                T v = T(0);
#pragma unroll
                for (int c = 0; c < NR; ++c) v = c == lane ? acc[r][c] : v;
                if (i0 + r < m && lane < nr) {
                    const T prev = beta == T(0) ? T(0) : beta * Cin[(i0 + r) * ldci + lane];
                    D[(i0 + r) * ldd + lane] = alpha * v + prev;
                }
            }
        }
    }
}

// op(A) = A, FP64, one contiguous right-hand side, 16-byte aligned rows of
// even length: the streaming form.  Each warp takes RW2 rows at a time; every
// lane loads 16-byte pairs of A and b, the loads of U column chunks issued
// together before their FMAs (RW2 x U + U pairs of 16 bytes in flight per
// lane), and the grid is one wave of CTAs resident on every SM.
template <int RW2, int U>
__global__ void __launch_bounds__(256) k_gemv_n2(int64_t m, int64_t k2, double alpha, const double2 *__restrict__ A,
                                                  int64_t lda2, const double2 *__restrict__ b, double beta,
                                                  const double *Cin, int64_t ldci, double *D, int64_t ldd,
                                                  const int *skip) {
    if (gemv_skipped(skip)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * 8;
    for (int64_t i0 = ((int64_t)blockIdx.x * 8 + warp) * RW2; i0 < m; i0 += nwarps * RW2) {
        const double2 *arow[RW2];
#pragma unroll
        for (int r = 0; r < RW2; ++r) arow[r] = A + (i0 + r < m ? i0 + r : i0) * lda2;
        double acc[RW2];
#pragma unroll
        for (int r = 0; r < RW2; ++r) acc[r] = 0.0;
        for (int64_t k0 = lane; k0 < k2; k0 += 32 * U) {
            double2 av[U][RW2], bv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t kk = k0 + 32 * u;
                const bool in = kk < k2;
                bv[u] = in ? __ldg(b + kk) : make_double2(0.0, 0.0);
#pragma unroll
                for (int r = 0; r < RW2; ++r) av[u][r] = in ? __ldcs(arow[r] + kk) : make_double2(0.0, 0.0);
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int r = 0; r < RW2; ++r) acc[r] = fma(av[u][r].y, bv[u].y, fma(av[u][r].x, bv[u].x, acc[r]));
        }
#pragma unroll
        for (int r = 0; r < RW2; ++r)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
        if (lane < RW2) {
            double v = 0.0;
#pragma unroll
            for (int r = 0; r < RW2; ++r) v = r == lane ? acc[r] : v;
            const int64_t i = i0 + lane;
            if (i < m) {
                const double prev = beta == 0.0 ? 0.0 : beta * Cin[i * ldci];
                D[i * ldd] = alpha * v + prev;
            }
        }
    }
}

template <typename T, int NR>
__global__ void __launch_bounds__(256) k_gemv_t(int64_t m, int nr, int64_t k, T alpha, const T *__restrict__ A,
                                                 int64_t lda, const T *__restrict__ B, int64_t ldb, T beta,
                                                 const T *Cin, int64_t ldci, T *D, int64_t ldd, const int *skip) {
    if (gemv_skipped(skip)) return;
    __shared__ T part[8][32][NR + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t j0 = (int64_t)blockIdx.x * 32; j0 < m; j0 += (int64_t)gridDim.x * 32) {
        const int64_t j = j0 + lane;
        const bool in = j < m;
        T acc[NR];
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] = T(0);
#pragma unroll 4
        for (int64_t kk = warp; kk < k; kk += 8) {
            const T a = in ? __ldg(A + kk * lda + j) : T(0);
#pragma unroll
            for (int c = 0; c < NR; ++c)
                if (c < nr) acc[c] = fma(a, __ldg(B + kk * ldb + c), acc[c]);
        }
#pragma unroll
        for (int c = 0; c < NR; ++c) part[warp][lane][c] = acc[c];
        __syncthreads();
        for (int idx = threadIdx.x; idx < 32 * nr; idx += 256) {
            const int l = idx / nr, c = idx % nr;
            const int64_t jj = j0 + l;
            if (jj < m) {
                T v = T(0);
#pragma unroll
                for (int w = 0; w < 8; ++w) v += part[w][l][c];
                const T prev = beta == T(0) ? T(0) : beta * Cin[jj * ldci + c];
                D[jj * ldd + c] = alpha * v + prev;
            }
        }
        __syncthreads();
    }
}

namespace {

template <typename T, int NR>
cudaError_t run_gemv(int64_t m, int64_t n, int64_t k, T alpha, const T *A, int64_t lda, bool transA, const T *B,
                     int64_t ldb, T beta, const T *Cin, int64_t ldci, T *D, int64_t ldd, const int *skip,
                     cudaStream_t s) {
    // algorithmic bytes: the m x k matrix read once
    auto *ev = profile_class_slot(kProfGemv, (double)m * (double)k * (double)sizeof(T));
    prof_begin(ev, s);
    note_launch();
    if (transA) {
        const int64_t blocks = cdiv(m, 32) < 65535 ? cdiv(m, 32) : 65535;
        k_gemv_t<T, NR><<<(unsigned)blocks, 256, 0, s>>>(m, (int)n, k, alpha, A, lda, B, ldb, beta, Cin, ldci, D,
                                                          ldd, skip);
    } else if (std::is_same<T, double>::value && n == 1 && ldb == 1 && k % 2 == 0 && lda % 2 == 0 &&
               (uintptr_t)A % 16 == 0 && (uintptr_t)B % 16 == 0) {
        // one contiguous RHS: 16-byte loads, four rows per warp, 8 x 16 B of A in
        // flight per lane, one wave of 8 CTAs per SM
        static int sms = 0;
        if (!sms) {
            int dev = 0;
            cudaGetDevice(&dev);
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 148;
        }
        constexpr int RW2 = 4, U = 2;
        const int64_t want = cdiv(m, 8 * RW2), blocks = want < 8 * sms ? want : 8 * sms;
        k_gemv_n2<RW2, U><<<(unsigned)blocks, 256, 0, s>>>(
            m, k / 2, (double)alpha, reinterpret_cast<const double2 *>(A), lda / 2,
            reinterpret_cast<const double2 *>(B), (double)beta, reinterpret_cast<const double *>(Cin), ldci,
            reinterpret_cast<double *>(D), ldd, skip);
    } else {
        // one RHS: two rows per warp, 16 loads in flight per lane and ~7 CTAs
        // per SM (the 4-row form left one wave of 3.4 CTAs per SM, 44% of HBM)
        constexpr int RW = NR == 1 ? 2 : (NR <= 4 ? 4 : 2);
        const int64_t blocks = cdiv(m, 8 * RW) < 65535 ? cdiv(m, 8 * RW) : 65535;
        k_gemv_n<T, NR, RW><<<(unsigned)blocks, 256, 0, s>>>(m, (int)n, k, alpha, A, lda, B, ldb, beta, Cin, ldci,
                                                              D, ldd, skip);
    }
    prof_end(ev, s);
    return cudaGetLastError();
}

template <typename T>
cudaError_t gemv(int64_t m, int64_t n, int64_t k, T alpha, const T *A, int64_t lda, bool transA, const T *B,
                 int64_t ldb, T beta, const T *Cin, int64_t ldci, T *D, int64_t ldd, const int *skip,
                 cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    if (n == 1) return run_gemv<T, 1>(m, n, k, alpha, A, lda, transA, B, ldb, beta, Cin, ldci, D, ldd, skip, s);
    if (n <= 2) return run_gemv<T, 2>(m, n, k, alpha, A, lda, transA, B, ldb, beta, Cin, ldci, D, ldd, skip, s);
    if (n <= 4) return run_gemv<T, 4>(m, n, k, alpha, A, lda, transA, B, ldb, beta, Cin, ldci, D, ldd, skip, s);
    if (n <= 8) return run_gemv<T, 8>(m, n, k, alpha, A, lda, transA, B, ldb, beta, Cin, ldci, D, ldd, skip, s);
    return run_gemv<T, 16>(m, n, k, alpha, A, lda, transA, B, ldb, beta, Cin, ldci, D, ldd, skip, s);
}

template <typename T, int BM, int BN, int BK, int TM, int TN, bool TA, int AS, int BS>
cudaError_t run(int64_t m, int64_t n, int64_t k, T alpha, const T *A, int64_t lda, const T *B, int64_t ldb,
                T beta, const T *Cin, int64_t ldci, T *D, int64_t ldd, const int *skip, const double *g,
                int64_t gn, cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    dim3 grid((unsigned)cdiv(n, BN), (unsigned)cdiv(m, BM));
    if (grid.y > 65535u) return cudaErrorInvalidValue;
    note_launch();
    k_gemm<T, BM, BN, BK, TM, TN, TA, AS, BS><<<grid, (BM / TM) * (BN / TN), 0, s>>>(
        m, n, k, alpha, A, lda, B, ldb, beta, Cin, ldci, D, ldd, skip, g, gn);
    return cudaGetLastError();
}

template <typename T, bool TA, int AS, int BS>
cudaError_t dispatch(int64_t m, int64_t n, int64_t k, T alpha, const T *A, int64_t lda, const T *B,
                     int64_t ldb, T beta, const T *Cin, int64_t ldci, T *D, int64_t ldd, const int *skip,
                     const double *g, int64_t gn, cudaStream_t s) {
    if (k < 0) k = 0;  // k == 0 gives D = beta * Cin
    if (n <= 16)
        return run<T, 64, 16, 16, 4, 4, TA, AS, BS>(m, n, k, alpha, A, lda, B, ldb, beta, Cin, ldci, D, ldd,
                                                     skip, g, gn, s);
    if (sizeof(T) == 8) {
        // FP64 is DFMA-bound: a product too small to give every SM two 64 x 64
        // tiles takes 32 x 32 tiles (four times the CTAs)
        if (cdiv(m, 64) * cdiv(n, 64) < 2 * 152)
            return run<T, 32, 32, 16, 2, 2, TA, AS, BS>(m, n, k, alpha, A, lda, B, ldb, beta, Cin, ldci, D, ldd,
                                                         skip, g, gn, s);
        return run<T, 64, 64, 16, 4, 4, TA, AS, BS>(m, n, k, alpha, A, lda, B, ldb, beta, Cin, ldci, D, ldd,
                                                     skip, g, gn, s);
    }
    return run<T, 128, 128, 8, 8, 8, TA, AS, BS>(m, n, k, alpha, A, lda, B, ldb, beta, Cin, ldci, D, ldd,
                                                  skip, g, gn, s);
}

}  // namespace

template <typename T>
cudaError_t gemm(int64_t m, int64_t n, int64_t k, T alpha, const T *A, int64_t lda, bool transA, const T *B,
                 int64_t ldb, T beta, const T *Cin, int64_t ldci, T *D, int64_t ldd, const int *skip,
                 cudaStream_t s) {
    // in-place updates (D == Cin) stay row-local in both skinny kernels: each
    // output entry reads its own Cin entry just before writing it
    if (n <= 16 && k > 0) return gemv<T>(m, n, k, alpha, A, lda, transA, B, ldb, beta, Cin, ldci, D, ldd, skip, s);
    if (transA)
        return dispatch<T, true, kDense, kDense>(m, n, k, alpha, A, lda, B, ldb, beta, Cin, ldci, D, ldd, skip,
                                                 nullptr, 1, s);
    return dispatch<T, false, kDense, kDense>(m, n, k, alpha, A, lda, B, ldb, beta, Cin, ldci, D, ldd, skip,
                                              nullptr, 1, s);
}

unsigned int gemv_skipped_count(bool reset) {
    unsigned int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_gemv_skipped, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (reset) {
        const unsigned int z = 0;
        cudaMemcpyToSymbol(g_gemv_skipped, &z, sizeof(z));
    }
    return v;
}

template cudaError_t gemm<double>(int64_t, int64_t, int64_t, double, const double *, int64_t, bool,
                                  const double *, int64_t, double, const double *, int64_t, double *, int64_t,
                                  const int *, cudaStream_t);
template cudaError_t gemm<float>(int64_t, int64_t, int64_t, float, const float *, int64_t, bool, const float *,
                                 int64_t, float, const float *, int64_t, float *, int64_t, const int *,
                                 cudaStream_t);

// C = A * G, G the leading n x n block of the circulant of order cn with
// first column g (cn = n: a circulant; cn = 2n: a Toeplitz matrix), any n:
// 2 n^3 operations.
template <typename TI, typename TO>
cudaError_t circ_matmul_direct(const double *g, int64_t cn, int64_t n, const TI *A, int64_t lda, TO *C, int64_t ldc,
                               cudaStream_t s) {
    static_assert(sizeof(TI) == sizeof(TO), "same precision in and out");
    return dispatch<TO, false, kDense, kCirc>(n, n, n, TO(1), (const TO *)A, lda, nullptr, 0, TO(0), nullptr, 0,
                                              C, ldc, nullptr, g, cn, s);
}
template cudaError_t circ_matmul_direct<double, double>(const double *, int64_t, int64_t, const double *, int64_t,
                                                        double *, int64_t, cudaStream_t);
template cudaError_t circ_matmul_direct<float, float>(const double *, int64_t, int64_t, const float *, int64_t,
                                                      float *, int64_t, cudaStream_t);

// X (+)= G Y or G^T Y for the same G without the DFT (any n).
cudaError_t circ_apply_direct(const double *g, int64_t cn, int64_t n, bool trans, const double *Y, int64_t ldy,
                              double *X, int64_t ldx, int64_t nrhs, bool accumulate, const int *skip, cudaStream_t s) {
    if (trans)
        return dispatch<double, false, kCircT, kDense>(n, nrhs, n, 1.0, nullptr, 0, Y, ldy, accumulate ? 1.0 : 0.0,
                                                       X, ldx, X, ldx, skip, g, cn, s);
    return dispatch<double, false, kCirc, kDense>(n, nrhs, n, 1.0, nullptr, 0, Y, ldy, accumulate ? 1.0 : 0.0, X,
                                                  ldx, X, ldx, skip, g, cn, s);
}

}  // namespace genp
