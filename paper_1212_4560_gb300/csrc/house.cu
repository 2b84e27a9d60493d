// house.cu -- products with the Householder multiplier H = I - 2 u u^T / n,
// u in {+-1}^n (the Householder multipliers of the tests cited in Sec. 7.1,
// read as an orthogonal reflector: u^T u = n).  H is symmetric, so
// H^T = H, and every product is a rank-one update:
//   C = A H = A - (2/n) (A u) u^T          (one CTA per row, the row read
//                                           twice, the second time from L2)
//   X = H Y = Y - (2/n) u (u^T Y)          (one CTA per right-hand side)
// HBM-bound: A read once, C written once.
#include "genp_internal.cuh"

namespace genp {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();                      // red is free
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    return t;
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(kThreads) k_house_rows(const double *u, int64_t n, double s, const TI *A,
                                                         int64_t lda, TO *C, int64_t ldc) {
    __shared__ double red[kThreads / 32];
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
        const TI *a = A + r * lda;
        double dot = 0.0;
        for (int64_t j = threadIdx.x; j < n; j += kThreads) dot = fma((double)a[j], u[j], dot);
        const double w = s * block_sum(dot, red);
        TO *c = C + r * ldc;
        for (int64_t j = threadIdx.x; j < n; j += kThreads) c[j] = (TO)fma(-w, u[j], (double)a[j]);
    }
}

__global__ void __launch_bounds__(kThreads) k_house_cols(const double *u, int64_t n, double s, const double *Y,
                                                         int64_t ldy, double *X, int64_t ldx, int accumulate,
                                                         const int *skip) {
    if (skip && *skip) return;
    __shared__ double red[kThreads / 32];
    const int64_t c = blockIdx.x;
    double dot = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kThreads) dot = fma(u[i], Y[i * ldy + c], dot);
    const double w = s * block_sum(dot, red);   // every read of Y is done (X may alias Y)
    for (int64_t i = threadIdx.x; i < n; i += kThreads) {
        const double v = fma(-w, u[i], Y[i * ldy + c]);
        X[i * ldx + c] = accumulate ? X[i * ldx + c] + v : v;
    }
}

// H[i][j] = delta_ij - (2 u_i u_j) / n, in that order of operations
__global__ void k_house_dense(const double *u, int64_t n, double *D, int64_t ldd) {
    for (int64_t i = blockIdx.y; i < n; i += gridDim.y)
        for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
            double v = 2.0 * u[i] * u[j];
            v = v / (double)n;
            D[i * ldd + j] = (i == j ? 1.0 : 0.0) - v;
        }
}

unsigned row_grid(int64_t n) { return (unsigned)(n < 152 * 8 ? n : 152 * 8); }

}  // namespace

template <typename TI, typename TO>
cudaError_t house_precondition(const genp_multiplier *G, const TI *A, int64_t lda, TO *C, int64_t ldc,
                               cudaStream_t s) {
    const int64_t n = G->n;
    note_launch();
    k_house_rows<TI, TO><<<row_grid(n), kThreads, 0, s>>>(G->g, n, 2.0 / (double)n, A, lda, C, ldc);
    return cudaGetLastError();
}
template cudaError_t house_precondition<double, double>(const genp_multiplier *, const double *, int64_t, double *,
                                                        int64_t, cudaStream_t);
template cudaError_t house_precondition<double, float>(const genp_multiplier *, const double *, int64_t, float *,
                                                       int64_t, cudaStream_t);
template cudaError_t house_precondition<float, float>(const genp_multiplier *, const float *, int64_t, float *,
                                                      int64_t, cudaStream_t);

cudaError_t house_apply(const genp_multiplier *G, const double *Y, int64_t ldy, double *X, int64_t ldx,
                        int64_t nrhs, bool accumulate, const int *skip, cudaStream_t s) {
    if (nrhs <= 0) return cudaSuccess;
    if (nrhs > 65535) return cudaErrorInvalidValue;
    note_launch();
    k_house_cols<<<(unsigned)nrhs, kThreads, 0, s>>>(G->g, G->n, 2.0 / (double)G->n, Y, ldy, X, ldx,
                                                     accumulate ? 1 : 0, skip);
    return cudaGetLastError();
}

cudaError_t house_to_dense(const genp_multiplier *G, double *D, int64_t ldd, cudaStream_t s) {
    const int64_t n = G->n;
    note_launch();
    k_house_dense<<<dim3((unsigned)cdiv(n < 2048 ? n : 2048, 256), (unsigned)(n < 65535 ? n : 65535)), 256, 0, s>>>(
        G->g, n, D, ldd);
    return cudaGetLastError();
}

}  // namespace genp
