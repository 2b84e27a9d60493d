// mixed.cu -- operands of the tensor-core products in mixed precision.
//
// A value x (FP32 or FP64) is split into BF16 terms
//   h1 = bf16(x),  h2 = bf16(x - h1),  h3 = bf16(x - h1 - h2)
// (each difference is exact in the source precision), so x = h1 + h2 + h3
// up to about 2^-24 |x|.  A product sum_k a_k b_k is then taken as
//   one term   (GENP_BF16):   a1 b1
//   six terms  (GENP_BF16X3): a1 b1 + a1 b2 + a2 b1 + a1 b3 + a2 b2 + a3 b1
// by laying the terms side by side along K:  A' = [a_t1 | a_t2 | ...],
// B' = [b_u1 | b_u2 | ...]; one BF16 GEMM over K' = terms * K then
// accumulates every product in FP32 on the tensor cores.  B' is written
// transposed (row j of B'^T holds column j of B), the K-major layout the
// tensor-core GEMM reads.
#include "genp_internal.cuh"

namespace genp {
namespace {

template <typename T>
__device__ __forceinline__ __nv_bfloat16 term(T x, int t) {
    __nv_bfloat16 h = __float2bfloat16_rn((float)x);
    for (int i = 0; i < t; ++i) {
        x = x - (T)__bfloat162float(h);
        h = __float2bfloat16_rn((float)x);
    }
    return h;
}

struct Pattern {
    int n;
    int t[6];
};

// dst[i][b*k + kk] = term_{p.t[b]}(src[i][kk]),  i < m, kk < k
template <typename T>
__global__ void k_split_rows(const T *src, int64_t lds, int64_t m, int64_t k, __nv_bfloat16 *dst, int64_t ldq,
                             Pattern p) {
    for (int64_t i = blockIdx.y; i < m; i += gridDim.y)
        for (int64_t kk = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; kk < k;
             kk += (int64_t)gridDim.x * blockDim.x) {
            const T x = src[i * lds + kk];
            for (int b = 0; b < p.n; ++b) dst[i * ldq + b * k + kk] = term(x, p.t[b]);
        }
}

// dst[j][b*k + kk] = term_{p.t[b]}(src[kk][j]),  kk < k, j < m   (32 x 32 tiles through shared memory)
template <typename T>
__global__ void k_split_cols_T(const T *src, int64_t lds, int64_t k, int64_t m, __nv_bfloat16 *dst, int64_t ldq,
                               Pattern p) {
    __shared__ T tile[32][33];
    const int64_t kk0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        const int64_t kk = kk0 + r, j = j0 + tx;
        tile[r][tx] = (kk < k && j < m) ? src[kk * lds + j] : T(0);
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t j = j0 + r, kk = kk0 + tx;
        if (j < m && kk < k) {
            const T x = tile[tx][r];
            for (int b = 0; b < p.n; ++b) dst[j * ldq + b * k + kk] = term(x, p.t[b]);
        }
    }
}

Pattern pattern_for(int terms, bool left) {
    Pattern p{};
    if (terms == 1) {
        p.n = 1;
        p.t[0] = 0;
    } else {
        static const int a[6] = {0, 0, 1, 0, 1, 2}, b[6] = {0, 1, 0, 2, 1, 0};
        p.n = 6;
        for (int i = 0; i < 6; ++i) p.t[i] = left ? a[i] : b[i];
    }
    return p;
}

}  // namespace

int split_terms(genp_prec p) { return p == GENP_BF16X3 ? 6 : 1; }

template <typename T>
cudaError_t split_rows(const T *src, int64_t lds, int64_t m, int64_t k, __nv_bfloat16 *dst, int64_t ldq, int terms,
                       bool left, int single_term, cudaStream_t s) {
    if (m <= 0 || k <= 0) return cudaSuccess;
    Pattern p = pattern_for(terms, left);
    if (single_term >= 0) {
        p.n = 1;
        p.t[0] = single_term;
    }
    dim3 g((unsigned)cdiv(k < 1024 ? k : 1024, 128), (unsigned)(m < 65535 ? m : 65535));
    note_launch();
    k_split_rows<T><<<g, 128, 0, s>>>(src, lds, m, k, dst, ldq, p);
    return cudaGetLastError();
}
template cudaError_t split_rows<float>(const float *, int64_t, int64_t, int64_t, __nv_bfloat16 *, int64_t, int, bool,
                                      int, cudaStream_t);
template cudaError_t split_rows<double>(const double *, int64_t, int64_t, int64_t, __nv_bfloat16 *, int64_t, int, bool,
                                       int, cudaStream_t);

template <typename T>
cudaError_t split_cols_T(const T *src, int64_t lds, int64_t k, int64_t m, __nv_bfloat16 *dst, int64_t ldq, int terms,
                         cudaStream_t s) {
    if (m <= 0 || k <= 0) return cudaSuccess;
    const Pattern p = pattern_for(terms, false);
    dim3 g((unsigned)cdiv(m, 32), (unsigned)cdiv(k, 32));
    if (g.y > 65535u) return cudaErrorInvalidValue;
    note_launch();
    k_split_cols_T<T><<<g, dim3(32, 8), 0, s>>>(src, lds, k, m, dst, ldq, p);
    return cudaGetLastError();
}
template cudaError_t split_cols_T<float>(const float *, int64_t, int64_t, int64_t, __nv_bfloat16 *, int64_t, int,
                                         cudaStream_t);

}  // namespace genp
