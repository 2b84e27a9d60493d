// solve.cu -- triangular solves with the GENP factors, refinement control
// and the adjoint's outer product.
//
// Solves are blocked by kBs rows: a one-CTA kernel solves the kBs x kBs
// diagonal triangle against all right-hand sides in shared memory, then a
// tiled GEMM subtracts that block's contribution from the remaining rows.
// The transposed pair (U^T then L^T) serves the adjoint (A^{-T} = L^{-T} U^{-T} G^T).
//
// Refinement (Sec. 7.1) is steered on the device: every iteration's kernels
// read a `done` flag that the stopping test sets, so a whole refinement is
// enqueued at once with no host synchronization.
#include "genp_internal.cuh"

#include <math.h>

namespace genp {
namespace {

constexpr int kBs = 64;
constexpr int kThreads = 256;
constexpr int kRhsTile = 32;

// mode 0: L (unit lower, forward)    mode 1: U (upper, backward)
// mode 2: U^T (lower, forward)       mode 3: L^T (unit upper, backward)
template <typename TS, typename T>
__global__ void __launch_bounds__(kThreads) k_diag_solve(const TS *C, int64_t ldc, int64_t b0, int bs, T *Y,
                                                         int64_t ldy, int nr, int mode, const int *skip) {
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *t = reinterpret_cast<T *>(smraw);          // bs x (bs+1): t[i][j] = op(C)[i][j]
    const int ld = bs + 1, tid = threadIdx.x;
    T *y = t + bs * ld;                           // bs x nr
    for (int idx = tid; idx < bs * bs; idx += kThreads) {
        const int i = idx / bs, j = idx % bs;
        const T v = (T)C[(b0 + i) * ldc + b0 + j];
        if (mode <= 1) t[i * ld + j] = v;
        else t[j * ld + i] = v;                   // transposed triangle
    }
    for (int idx = tid; idx < bs * nr; idx += kThreads) {
        const int i = idx / nr, c = idx % nr;
        y[i * nr + c] = Y[(b0 + i) * ldy + c];
    }
    __syncthreads();
    const bool forward = (mode == 0 || mode == 2);
    const bool unit = (mode == 0 || mode == 3);
    for (int s = 0; s < bs; ++s) {
        const int k = forward ? s : bs - 1 - s;
        if (!unit) {
            if (tid < nr) y[k * nr + tid] = y[k * nr + tid] / t[k * ld + k];
            __syncthreads();
        }
        const int lo = forward ? k + 1 : 0, hi = forward ? bs : k;
        const int cnt = (hi - lo) * nr;
        for (int idx = tid; idx < cnt; idx += kThreads) {
            const int i = lo + idx / nr, c = idx % nr;
            y[i * nr + c] = y[i * nr + c] - t[i * ld + k] * y[k * nr + c];
        }
        __syncthreads();
    }
    for (int idx = tid; idx < bs * nr; idx += kThreads) {
        const int i = idx / nr, c = idx % nr;
        Y[(b0 + i) * ldy + c] = y[i * nr + c];
    }
}

template <typename TS, typename TD>
__global__ void k_convert(const TS *src, int64_t lds, TD *dst, int64_t ldd, int64_t m, int64_t n, const int *skip) {
    if (skip && *skip) return;
    for (int64_t r = blockIdx.y; r < m; r += gridDim.y)
        for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
            dst[r * ldd + c] = (TD)src[r * lds + c];
}

// ||A||_inf = max_r sum_j |a_rj| (one warp per row).
__global__ void k_rownorm_inf(const double *A, int64_t lda, int64_t n, unsigned long long *out) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double best = 0.0;
    for (int64_t r = warp; r < n; r += nw) {
        double s = 0.0;
        for (int64_t j = lane; j < n; j += 32) s += fabs(A[r * lda + j]);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        best = (s > best || isnan(s)) ? s : best;
    }
    if (lane == 0) atomic_max_nonneg(out, best);
}

__global__ void k_refine_reset(DevStatus *st, DevNorms *nm, unsigned long long *anorm_bits) {
    st->refine_iters = 0;
    st->refine_done = 0;
    st->refine_status = GENP_OK;
    for (int i = 0; i <= GENP_MAX_REFINE; ++i) st->bwd_err[i] = -1.0;
    for (int c = 0; c < kMaxRhsChunk; ++c) nm->r[c] = nm->x[c] = nm->b[c] = 0ull;
    *anorm_bits = 0ull;
}

__global__ void k_anorm_store(DevStatus *st, const unsigned long long *anorm_bits) {
    st->anorm = __longlong_as_double((long long)*anorm_bits);
}

// Column-wise infinity norms of R, X and B (one thread per row, nrhs columns).
__global__ void k_colnorms(const double *R, int64_t ldr, const double *X, int64_t ldx, const double *B,
                           int64_t ldb, int64_t n, int nrhs, DevNorms *nm, const int *done) {
    if (*done) return;
    __shared__ double sr[kMaxRhsChunk], sx[kMaxRhsChunk], sb[kMaxRhsChunk];
    if (threadIdx.x < kMaxRhsChunk) sr[threadIdx.x] = sx[threadIdx.x] = sb[threadIdx.x] = 0.0;
    __syncthreads();
    double mr[kMaxRhsChunk], mx[kMaxRhsChunk], mb[kMaxRhsChunk];
    for (int c = 0; c < nrhs; ++c) mr[c] = mx[c] = mb[c] = 0.0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        for (int c = 0; c < nrhs; ++c) {
            const double a = fabs(R[r * ldr + c]), bx = fabs(X[r * ldx + c]), bb = fabs(B[r * ldb + c]);
            mr[c] = (a > mr[c] || isnan(a)) ? a : mr[c];
            mx[c] = (bx > mx[c] || isnan(bx)) ? bx : mx[c];
            mb[c] = (bb > mb[c] || isnan(bb)) ? bb : mb[c];
        }
    for (int c = 0; c < nrhs; ++c) {
        double a = mr[c], bx = mx[c], bb = mb[c];
        for (int o = 16; o > 0; o >>= 1) {
            const double u = __shfl_xor_sync(0xffffffffu, a, o), v = __shfl_xor_sync(0xffffffffu, bx, o),
                         w = __shfl_xor_sync(0xffffffffu, bb, o);
            a = (u > a || isnan(u)) ? u : a;
            bx = (v > bx || isnan(v)) ? v : bx;
            bb = (w > bb || isnan(w)) ? w : bb;
        }
        if ((threadIdx.x & 31) == 0) {
            atomic_max_nonneg((unsigned long long *)&sr[c], a);
            atomic_max_nonneg((unsigned long long *)&sx[c], bx);
            atomic_max_nonneg((unsigned long long *)&sb[c], bb);
        }
    }
    __syncthreads();
    if (threadIdx.x < nrhs) {
        atomic_max_nonneg(&nm->r[threadIdx.x], sr[threadIdx.x]);
        atomic_max_nonneg(&nm->x[threadIdx.x], sx[threadIdx.x]);
        atomic_max_nonneg(&nm->b[threadIdx.x], sb[threadIdx.x]);
    }
}

// Stopping test of refinement step `it` (it = 0: the unrefined solution).
__global__ void k_refine_decide(DevStatus *st, DevNorms *nm, int nrhs, int it, double tol, int max_iter) {
    if (st->refine_done) return;
    const double an = st->anorm;
    double eta = 0.0;
    for (int c = 0; c < nrhs; ++c) {
        const double r = __longlong_as_double((long long)nm->r[c]);
        const double x = __longlong_as_double((long long)nm->x[c]);
        const double b = __longlong_as_double((long long)nm->b[c]);
        double e = r / (an * x + b);
        if (!(e == e)) e = INFINITY;
        eta = e > eta ? e : eta;
        nm->r[c] = nm->x[c] = nm->b[c] = 0ull;
    }
    st->bwd_err[it] = eta;
    st->refine_iters = it;
    const bool stagnated = it > 0 && eta > 0.5 * st->bwd_err[it - 1];
    if (eta <= tol) {
        st->refine_done = 1;
        st->refine_status = GENP_OK;
    } else if (stagnated || it >= max_iter) {
        st->refine_done = 1;
        st->refine_status = GENP_ERR_NOCONV;
    }
}

// dA[i][j] = - sum_c Lam[i][c] X[j][c]   (32 x 32 output tile per CTA)
template <typename TD>
__global__ void k_outer(const double *Lam, int64_t ldl, const double *X, int64_t ldx, int64_t n, int nrhs, TD *dA,
                        int64_t ldda) {
    __shared__ double sl[32][kMaxRhsChunk + 1], sxx[32][kMaxRhsChunk + 1];
    const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
    double acc[4] = {0, 0, 0, 0};
    for (int c0 = 0; c0 < nrhs; c0 += kMaxRhsChunk) {
        const int cw = min(kMaxRhsChunk, nrhs - c0);
        __syncthreads();
        for (int idx = threadIdx.x; idx < 32 * cw; idx += blockDim.x) {
            const int r = idx / cw, c = idx % cw;
            sl[r][c] = (i0 + r < n) ? Lam[(i0 + r) * ldl + c0 + c] : 0.0;
            sxx[r][c] = (j0 + r < n) ? X[(j0 + r) * ldx + c0 + c] : 0.0;
        }
        __syncthreads();
        for (int q = 0; q < 4; ++q) {
            const int r = ty + 8 * q;
            double s = 0.0;
            for (int c = 0; c < cw; ++c) s = fma(sl[r][c], sxx[tx][c], s);
            acc[q] += s;
        }
    }
    for (int q = 0; q < 4; ++q) {
        const int64_t i = i0 + ty + 8 * q, j = j0 + tx;
        if (i < n && j < n) dA[i * ldda + j] = (TD)(-acc[q]);
    }
}

template <typename TS, typename T>
cudaError_t solve_typed(const genp_factors *F, T *Y, int64_t ldy, int64_t nrhs, bool transposed, const int *skip,
                        cudaStream_t s) {
    const TS *C = static_cast<const TS *>(F->C);
    const int64_t n = F->n, ldc = F->ldc;
    const int64_t nblk = cdiv(n, kBs);
    static bool attr_done = false;
    if (!attr_done) {
        cudaFuncSetAttribute(k_diag_solve<TS, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
        attr_done = true;
    }
    for (int64_t c0 = 0; c0 < nrhs; c0 += kRhsTile) {
        const int nr = (int)(nrhs - c0 < kRhsTile ? nrhs - c0 : kRhsTile);
        T *Yc = Y + c0;
        for (int pass = 0; pass < 2; ++pass) {
            // pass 0: L (or U^T) forward; pass 1: U (or L^T) backward
            const int mode = transposed ? (pass == 0 ? 2 : 3) : (pass == 0 ? 0 : 1);
            for (int64_t q = 0; q < nblk; ++q) {
                const int64_t blk = pass == 0 ? q : nblk - 1 - q;
                const int64_t b0 = blk * kBs;
                const int bs = (int)(n - b0 < kBs ? n - b0 : kBs);
                const size_t sm = ((size_t)bs * (bs + 1) + (size_t)bs * nr) * sizeof(T);
                note_launch();
                k_diag_solve<TS, T><<<1, kThreads, sm, s>>>(C, ldc, b0, bs, Yc, ldy, nr, mode, skip);
                cudaError_t e;
                if (pass == 0) {
                    const int64_t r0 = b0 + bs, rem = n - r0;
                    if (rem <= 0) continue;
                    // rows below: Y[r0:] -= op(C)[r0:, b0:b0+bs] * Y[b0:b0+bs]
                    if (!transposed)
                        e = gemm<T>(rem, nr, bs, T(-1), (const T *)(C + r0 * ldc + b0), ldc, false, Yc + b0 * ldy, ldy,
                                    T(1), Yc + r0 * ldy, ldy, Yc + r0 * ldy, ldy, skip, s);
                    else  // (U^T)[r0+i][b0+k] = U[b0+k][r0+i]
                        e = gemm<T>(rem, nr, bs, T(-1), (const T *)(C + b0 * ldc + r0), ldc, true, Yc + b0 * ldy, ldy,
                                    T(1), Yc + r0 * ldy, ldy, Yc + r0 * ldy, ldy, skip, s);
                } else {
                    const int64_t rem = b0;
                    if (rem <= 0) continue;
                    if (!transposed)  // U[0:b0, b0:b0+bs]
                        e = gemm<T>(rem, nr, bs, T(-1), (const T *)(C + b0), ldc, false, Yc + b0 * ldy, ldy, T(1), Yc,
                                    ldy, Yc, ldy, skip, s);
                    else  // (L^T)[i][b0+k] = L[b0+k][i]
                        e = gemm<T>(rem, nr, bs, T(-1), (const T *)(C + b0 * ldc), ldc, true, Yc + b0 * ldy, ldy, T(1),
                                    Yc, ldy, Yc, ldy, skip, s);
                }
                if (e != cudaSuccess) return e;
            }
        }
    }
    return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t lu_solve_inplace(const genp_factors *F, T *Y, int64_t ldy, int64_t nrhs, bool transposed, const int *skip,
                             cudaStream_t s) {
    if (sizeof(T) == 8) {
        if (F->prec != GENP_FP64) return cudaErrorInvalidValue;
        return solve_typed<T, T>(F, Y, ldy, nrhs, transposed, skip, s);
    }
    if (F->prec == GENP_FP64) return cudaErrorInvalidValue;
    return solve_typed<float, T>(F, Y, ldy, nrhs, transposed, skip, s);
}
template cudaError_t lu_solve_inplace<double>(const genp_factors *, double *, int64_t, int64_t, bool, const int *,
                                              cudaStream_t);
template cudaError_t lu_solve_inplace<float>(const genp_factors *, float *, int64_t, int64_t, bool, const int *,
                                             cudaStream_t);

template <typename TS, typename TD>
cudaError_t convert_matrix(const TS *src, int64_t lds, TD *dst, int64_t ldd, int64_t m, int64_t n, const int *skip,
                           cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    dim3 g((unsigned)cdiv(n < 256 ? n : 256, 256), (unsigned)(m < 65535 ? m : 65535));
    note_launch();
    k_convert<TS, TD><<<g, 256, 0, s>>>(src, lds, dst, ldd, m, n, skip);
    return cudaGetLastError();
}
template cudaError_t convert_matrix<double, float>(const double *, int64_t, float *, int64_t, int64_t, int64_t,
                                                   const int *, cudaStream_t);
template cudaError_t convert_matrix<float, double>(const float *, int64_t, double *, int64_t, int64_t, int64_t,
                                                   const int *, cudaStream_t);
template cudaError_t convert_matrix<double, double>(const double *, int64_t, double *, int64_t, int64_t, int64_t,
                                                    const int *, cudaStream_t);
template cudaError_t convert_matrix<float, float>(const float *, int64_t, float *, int64_t, int64_t, int64_t,
                                                  const int *, cudaStream_t);

cudaError_t refine_init(genp_factors *F, const double *A, int64_t lda, int64_t n, cudaStream_t s) {
    unsigned long long *bits = reinterpret_cast<unsigned long long *>(&F->norms[1]);
    note_launch();
    k_refine_reset<<<1, 1, 0, s>>>(F->st, F->norms, bits);
    note_launch();
    k_rownorm_inf<<<152 * 4, 256, 0, s>>>(A, lda, n, bits);
    note_launch();
    k_anorm_store<<<1, 1, 0, s>>>(F->st, bits);
    return cudaGetLastError();
}

cudaError_t refine_check(genp_factors *F, const double *R, int64_t ldr, const double *X, int64_t ldx, const double *B,
                         int64_t ldb, int64_t n, int64_t nrhs, int it, double tol, int max_iter, int, cudaStream_t s) {
    if (nrhs > kMaxRhsChunk) return cudaErrorInvalidValue;
    note_launch();
    k_colnorms<<<152 * 2, 256, 0, s>>>(R, ldr, X, ldx, B, ldb, n, (int)nrhs, F->norms, &F->st->refine_done);
    note_launch();
    k_refine_decide<<<1, 1, 0, s>>>(F->st, F->norms, (int)nrhs, it, tol, max_iter);
    return cudaGetLastError();
}

cudaError_t outer_update(const double *Lam, int64_t ldl, const double *X, int64_t ldx, int64_t n, int64_t nrhs,
                         void *dA, int64_t ldda, bool dA_f32, cudaStream_t s) {
    dim3 g((unsigned)cdiv(n, 32), (unsigned)cdiv(n, 32));
    if (dA_f32) {
        note_launch();
        k_outer<float><<<g, 256, 0, s>>>(Lam, ldl, X, ldx, n, (int)nrhs, (float *)dA, ldda);
    } else {
        note_launch();
        k_outer<double><<<g, 256, 0, s>>>(Lam, ldl, X, ldx, n, (int)nrhs, (double *)dA, ldda);
    }
    return cudaGetLastError();
}

}  // namespace genp
