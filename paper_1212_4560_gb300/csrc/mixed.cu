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

#include <cuda_fp8.h>

#include "e4m3.cuh"

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

// ---------------------------------------------------------------------------
// E4M3 operands with a power-of-two scale per 128 x 128 tile.  For the
// logical operand X (m x K; X[i][k] = src[i lds + k], or src[k lds + i] when
// the source is stored transposed) tile (ti, kt) gets the scale 2^e with e
// the least integer such that max |X_tile| <= 448 2^e (448: the largest
// finite e4m3 value), clamped to [-126, 126] so the scale is a normal float
// (e = 0 for an all-zero tile).  With max |X_tile| = f 2^p, f in [0.5, 1):
// e = p - 9 when f <= 0.875, else p - 8.  Then
//   dst[i ldq + k] = e4m3_rn_satfinite(X[i][k] 2^-e),  scales[ti nkt + kt] = 2^e
// (the product X 2^-e is exact).  One CTA of 256 threads per tile.
// ---------------------------------------------------------------------------
constexpr int QT = 128;

__device__ __forceinline__ uint8_t to_e4m3(float v) {
    return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}
__device__ __forceinline__ uint8_t to_e4m3(double v) { return e4m3_code_f64(v); }
template <typename T>
__device__ __forceinline__ T pow2_of(int k);
template <>
__device__ __forceinline__ float pow2_of<float>(int k) { return __int_as_float((127 + k) << 23); }
template <>
__device__ __forceinline__ double pow2_of<double>(int k) { return __longlong_as_double((long long)(1023 + k) << 52); }
// |x| as an integer key whose order is that of the magnitudes (non-negative
// IEEE values order like their bit patterns): the tile maximum without FP64 work
__device__ __forceinline__ unsigned long long mag_key(float v) { return __float_as_uint(v) & 0x7FFFFFFFu; }
__device__ __forceinline__ unsigned long long mag_key(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ double key_value(unsigned long long k, float) { return (double)__uint_as_float((uint32_t)k); }
__device__ __forceinline__ double key_value(unsigned long long k, double) { return __longlong_as_double((long long)k); }
__device__ __forceinline__ int tile_exponent(double amax) {
    if (!(amax > 0.0) || !isfinite(amax)) return 0;
    int p = 0;
    const double f = frexp(amax, &p);
    int e = f <= 0.875 ? p - 9 : p - 8;
    return e < -126 ? -126 : (e > 126 ? 126 : e);
}

template <typename T, bool TRANS>
__global__ void __launch_bounds__(256) k_quant_e4m3(const T *__restrict__ src, int64_t lds, int m, int K,
                                                    uint8_t *__restrict__ dst, int64_t ldq, float *scales, int nkt) {
    __shared__ unsigned long long red[8];
    __shared__ int s_e;
    __shared__ __align__(16) uint8_t qt[TRANS ? QT : 1][QT + 4];   // transposed tile (i, k)
    const int kt = blockIdx.x, ti = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i0 = ti * QT, k0 = kt * QT;
    // the tile as 128 source rows r of 128 contiguous source elements c
    const int R = TRANS ? K : m, CC = TRANS ? m : K;
    const int r0 = TRANS ? k0 : i0, c0 = TRANS ? i0 : k0;
    // two passes over the tile (the second mostly from L1/L2): source rows
    // warp + 8 i, elements lane + 32 j, coalesced along rows
    unsigned long long amax = 0;
#pragma unroll 4
    for (int i = 0; i < 16; ++i) {
        const int r = warp + 8 * i;
        if (r0 + r >= R) break;
        const T *row = src + (int64_t)(r0 + r) * lds + c0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = lane + 32 * j;
            if (c0 + c < CC) amax = max(amax, mag_key(row[c]));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (lane == 0) red[warp] = amax;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long a = red[0];
        for (int w = 1; w < 8; ++w) a = max(a, red[w]);
        const int e = tile_exponent(key_value(a, T(0)));
        s_e = e;
        scales[(int64_t)ti * nkt + kt] = ldexpf(1.0f, e);
    }
    __syncthreads();
    const int e = s_e;
    const T down = pow2_of<T>(-e);   // exact: |e| <= 126
#pragma unroll 4
    for (int i = 0; i < 16; ++i) {
        const int r = warp + 8 * i;
        if (r0 + r >= R) break;
        const T *row = src + (int64_t)(r0 + r) * lds + c0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = lane + 32 * j;
            const uint8_t q = c0 + c < CC ? to_e4m3(row[c] * down) : (uint8_t)0;
            if (TRANS) qt[c][r] = q;
            else if (c0 + c < CC) dst[(int64_t)(r0 + r) * ldq + c0 + c] = q;
        }
    }
    if (TRANS) {
        __syncthreads();
        // dst row i0 + cc holds k0 .. k0 + 127 (the source rows)
        const int c = lane * 4;
        for (int cc = warp; cc < QT && i0 + cc < m; cc += 8) {
            uint8_t *d = dst + (int64_t)(i0 + cc) * ldq + k0 + c;
            if (k0 + c + 3 < K) {
                *reinterpret_cast<uint32_t *>(d) = *reinterpret_cast<const uint32_t *>(&qt[cc][c]);
            } else {
                for (int j = 0; j < 4 && k0 + c + j < K; ++j) d[j] = qt[cc][c + j];
            }
        }
    }
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

namespace genp {

int64_t e4m3_tiles(int64_t rows, int64_t K) { return cdiv(rows, QT) * cdiv(K, QT); }

template <typename T>
cudaError_t quant_e4m3(const T *src, int64_t lds, int64_t m, int64_t K, bool trans, uint8_t *dst, int64_t ldq,
                       float *scales, cudaStream_t s) {
    if (m <= 0 || K <= 0) return cudaSuccess;
    if (m > INT32_MAX || K > INT32_MAX || ldq < K || (ldq % 4) || ((uintptr_t)dst % 4)) return cudaErrorInvalidValue;
    const int64_t nkt = cdiv(K, QT), ntm = cdiv(m, QT);
    if (nkt > INT32_MAX || ntm > 65535) return cudaErrorInvalidValue;
    dim3 g((unsigned)nkt, (unsigned)ntm);
    note_launch();
    if (trans)
        k_quant_e4m3<T, true><<<g, 256, 0, s>>>(src, lds, (int)m, (int)K, dst, ldq, scales, (int)nkt);
    else
        k_quant_e4m3<T, false><<<g, 256, 0, s>>>(src, lds, (int)m, (int)K, dst, ldq, scales, (int)nkt);
    return cudaGetLastError();
}
template cudaError_t quant_e4m3<float>(const float *, int64_t, int64_t, int64_t, bool, uint8_t *, int64_t, float *,
                                       cudaStream_t);
template cudaError_t quant_e4m3<double>(const double *, int64_t, int64_t, int64_t, bool, uint8_t *, int64_t, float *,
                                        cudaStream_t);

}  // namespace genp
