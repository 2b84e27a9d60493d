// sparse.cu -- products with the sparse +-1 multiplier G = sum_t D_t P_t.
//
// Column j of G holds signs[t][j] at row rows[t][j], t < nnz, so
//   (A G)[r][j] = sum_t signs[t][j] * A[r][rows[t][j]]          (a signed gather)
//   (G Y)[i]    = sum_t inv_signs[t][i] * Y[inv_rows[t][i]]     (inverse permutations)
//   (G^T Y)[j]  = sum_t signs[t][j] * Y[rows[t][j]]
// These are memory-bound: A G reads A once and writes C once.  One CTA
// handles one row of A at a time, staged in shared memory so that the
// random gathers hit on-chip memory; the index arrays stay in L2.
#include "genp_internal.cuh"

namespace genp {
namespace {

constexpr int kThreads = 512;
constexpr int64_t kMaxSmemRow = 96 * 1024;

template <typename TI, typename TO, bool SMEM>
__global__ void __launch_bounds__(kThreads)
k_sparse_pre(const int32_t *__restrict__ rows, const int8_t *__restrict__ signs, int64_t n, int nnz,
             const TI *__restrict__ A, int64_t lda, TO *__restrict__ C, int64_t ldc) {
    extern __shared__ __align__(16) unsigned char smraw[];
    TI *row = reinterpret_cast<TI *>(smraw);
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
        const TI *a = A + r * lda;
        if (SMEM) {
            __syncthreads();
            for (int64_t j = threadIdx.x; j < n; j += blockDim.x) row[j] = a[j];
            __syncthreads();
        }
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
            TO s = TO(0);
            for (int t = 0; t < nnz; ++t) {
                const int64_t src = rows[(int64_t)t * n + j];
                const TO v = (TO)(SMEM ? row[src] : a[src]);
                s = signs[(int64_t)t * n + j] > 0 ? s + v : s - v;
            }
            C[r * ldc + j] = s;
        }
    }
}

__global__ void k_sparse_apply(const int32_t *__restrict__ idx, const int8_t *__restrict__ sg, int64_t n, int nnz,
                               const double *__restrict__ Y, int64_t ldy, double *X, int64_t ldx, int nrhs,
                               int accumulate, const int *skip) {
    if (skip && *skip) return;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nrhs; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / nrhs, c = e % nrhs;
        double s = 0.0;
        for (int t = 0; t < nnz; ++t) {
            const double v = Y[(int64_t)idx[(int64_t)t * n + i] * ldy + c];
            s = sg[(int64_t)t * n + i] > 0 ? s + v : s - v;
        }
        X[i * ldx + c] = accumulate ? X[i * ldx + c] + s : s;
    }
}

}  // namespace

template <typename TI, typename TO>
cudaError_t sparse_precondition(const genp_multiplier *G, const TI *A, int64_t lda, TO *C, int64_t ldc,
                                cudaStream_t s) {
    const int64_t n = G->n;
    const int blocks = (int)(n < 152 * 8 ? n : 152 * 8);
    const size_t sm = (size_t)n * sizeof(TI);
    if ((int64_t)sm <= kMaxSmemRow) {
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_sparse_pre<TI, TO, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kMaxSmemRow);
            attr = true;
        }
        note_launch();
        k_sparse_pre<TI, TO, true><<<blocks, kThreads, sm, s>>>(G->rows, G->signs, n, G->nnz, A, lda, C, ldc);
    } else {
        note_launch();
        k_sparse_pre<TI, TO, false><<<blocks, kThreads, 0, s>>>(G->rows, G->signs, n, G->nnz, A, lda, C, ldc);
    }
    return cudaGetLastError();
}
template cudaError_t sparse_precondition<double, double>(const genp_multiplier *, const double *, int64_t, double *,
                                                         int64_t, cudaStream_t);
template cudaError_t sparse_precondition<float, float>(const genp_multiplier *, const float *, int64_t, float *,
                                                       int64_t, cudaStream_t);
template cudaError_t sparse_precondition<double, float>(const genp_multiplier *, const double *, int64_t, float *,
                                                        int64_t, cudaStream_t);

cudaError_t sparse_apply(const genp_multiplier *G, bool trans, const double *Y, int64_t ldy, double *X, int64_t ldx,
                         int64_t nrhs, bool accumulate, const int *skip, cudaStream_t s) {
    const int64_t n = G->n;
    const int64_t work = n * nrhs;
    int blocks = (int)cdiv(work, 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    if (trans) {
        note_launch();
        k_sparse_apply<<<blocks, 256, 0, s>>>(G->rows, G->signs, n, G->nnz, Y, ldy, X, ldx, (int)nrhs, accumulate, skip);
    } else {
        note_launch();
        k_sparse_apply<<<blocks, 256, 0, s>>>(G->inv_rows, G->inv_signs, n, G->nnz, Y, ldy, X, ldx, (int)nrhs,
                                              accumulate, skip);
    }
    return cudaGetLastError();
}

}  // namespace genp
