// sliced.cu -- FP64-class products on the BF16 tensor cores by exact
// fixed-point slicing (the Ozaki scheme: Ozaki, Ogita, Oishi & Rump,
// "Error-free transformations of matrix multiplication", Numer. Algorithms
// 2012).  The digit layout and the accumulator groups are in sliced.cuh; this
// file cuts FP64 operands into their BF16 digit slices, and holds the
// double-float helpers of the GENP_BF16_SLICED factorization.
//
// With ND digits the kept pairs (t + u <= ND + 1) and the truncation leave at
// most about 2^-(7 ND - 1) of 2^{e_i + f_j} per term of the sum over k, and
// every digit group but the last is summed exactly (K <= 512).
#include "genp_internal.cuh"
#include "dfloat.cuh"
#include "sliced.cuh"

#include <math.h>

namespace genp {

namespace {

int g_default_digits = 7;
int g_precond_digits = 7;
int g_mult_digits = 1;

// An operand entry in FP64: the double-float trailing matrix of the sliced
// factorization converts exactly (48 significant bits).
__device__ __forceinline__ double as_f64(double x) { return x; }
__device__ __forceinline__ double as_f64(dfloat v) { return (double)v.hi + (double)v.lo; }

// |x| as its IEEE bit pattern, NaN mapped to 0: the integer maximum of these
// is the bit pattern of max|x| (no FP64 min/max on the scarce FP64 units)
__device__ __forceinline__ unsigned long long abs_bits(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
    return b > 0x7FF0000000000000ull ? 0ull : b;
}

// exponent e with max|x| < 2^e (0 for an all-zero row)
__device__ __forceinline__ int scale_exp(double amax) {
    if (!(amax > 0.0)) return 0;
    int e;
    frexp(amax, &e);   // amax = m 2^e, m in [0.5, 1)
    return e;
}

// Ordering key of |x| 2^sc from the IEEE bit pattern (integer work only):
// the biased exponent moved by sc in 12 bits above the mantissa, so the
// integer maximum of keys is the key of max |x| 2^sc.  Zero and subnormal
// x give 0 (too small to set a scale), NaN gives 0, infinity the largest key.
__device__ __forceinline__ unsigned long long scaled_key(double x, int sc) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
    if (b > 0x7FF0000000000000ull) return 0ull;
    const int E = (int)(b >> 52);
    if (E == 0) return 0ull;
    if (E == 0x7FF) return ~0ull;
    int t = E + sc;
    t = t < -2047 ? -2047 : (t > 2047 ? 2047 : t);
    return ((unsigned long long)(t + 2048) << 52) | (b & 0xFFFFFFFFFFFFFull);
}

// exponent e with max|x| 2^sc < 2^e from the maximum key (0 for none)
__device__ __forceinline__ int key_exp(unsigned long long key) {
    if (key == 0ull) return 0;
    if (key == ~0ull) return 2047;
    return (int)(key >> 52) - 2048 - 1022;
}

// Digits of q = x 2^-e in (-1, 1): X = round(q 2^(7 ND)) (an integer below
// 2^(7 ND) in magnitude), then its balanced base-128 digits from the
// bottom: d_t = ((X + 64) mod 128) - 64 in [-64, 63], X <- (X - d_t) / 128;
// what is left is d_1 in [-128, 128].  X comes straight from the IEEE bit
// pattern (x = mant 2^ex, shifted by ex + 7 ND - e with round-half-even),
// all in integer arithmetic: GB300's FP64 units, where scaling and
// conversion would run, are scarce.  The dropped remainder is below
// 2^-(7 ND + 1); a non-finite x gives X = 0.
template <int ND>
__device__ __forceinline__ void digits(double x, int e, float (&d)[ND], int sc = 0) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
    int ex = -1074;                                   // x = mant 2^ex
    if (E != 0) {
        mant |= 1ull << 52;
        ex = E - 1075;
    }
    const int sh = ex + sc + 7 * ND - e;            // x 2^sc scaled by 2^-e
    unsigned long long m = 0;
    if (E == 0x7FF || mant == 0) {
        m = 0;
    } else if (sh >= 0) {
        m = mant << sh;                               // below 2^(7 ND): |x| < 2^e
    } else if (sh > -64) {
        const int r = -sh;
        const unsigned long long q = mant >> r, rem = mant & ((1ull << r) - 1), half = 1ull << (r - 1);
        m = q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
    }
    long long X = (b >> 63) ? -(long long)m : (long long)m;
#pragma unroll
    for (int t = ND - 1; t >= 1; --t) {
        const long long lo = ((X + 64) & 127) - 64;
        d[t] = (float)(int)lo;
        X = (X - lo) >> 7;
    }
    d[0] = (float)(int)X;
}

// Writes the ND digit slices of one operand entry (a small integer each: exact in BF16).
template <int ND>
__device__ __forceinline__ void put(__nv_bfloat16 *row, int64_t kpad, int64_t k, const float (&d)[ND]) {
#pragma unroll
    for (int t = 0; t < ND; ++t) row[t * kpad + k] = __float2bfloat16_rn(d[t]);
}

// A operand: rows of src (m x K, FP64 or double-float, ld lds).  One warp
// per row.  With kexp, entry k of every row is taken as x 2^-kexp[k] (an
// exact power-of-two scaling of the inner dimension that the B operand
// undoes; see slice_cols_T).
template <int ND, typename TS>
__global__ void k_slice_rows(const TS *src, int64_t lds, int64_t m, int64_t K, int64_t kpad,
                             __nv_bfloat16 *dst, int64_t ldq, int *exps, const unsigned long long *kkey) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < m; i += nw) {
        const TS *a = src + i * lds;
        int e;
        unsigned long long mb = 0ull;
        if (kkey) {
            for (int64_t k = lane; k < K; k += 32) mb = max(mb, scaled_key(as_f64(a[k]), -key_exp(kkey[k])));
            for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
            e = key_exp(mb);
        } else {
            for (int64_t k = lane; k < K; k += 32) mb = max(mb, abs_bits(as_f64(a[k])));
            for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
            e = scale_exp(__longlong_as_double((long long)mb));
        }
        if (lane == 0) exps[i] = e;
        __nv_bfloat16 *row = dst + i * ldq;
        for (int64_t k = lane; k < kpad; k += 32) {
            float d[ND] = {};
            if (k < K) digits<ND>(as_f64(a[k]), e, d, kkey ? -key_exp(kkey[k]) : 0);
            put<ND>(row, kpad, k, d);
        }
    }
}

// B operand: columns of src (K x n, FP64, ld lds), written transposed
// (row j of dst holds column j).  Pass 1: column exponents; a CTA takes 32
// columns, its 8 warps split the rows (coalesced 256-byte rows per warp),
// and the 8 partial maxima meet in shared memory.
// With kkey, row k of src is taken as x 2^+q_k, q_k = key_exp(kkey[k]).
template <typename TS>
__global__ void k_col_exps(const TS *src, int64_t lds, int64_t K, int64_t n, int *exps,
                           const unsigned long long *kkey) {
    __shared__ unsigned long long part[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t j = (int64_t)blockIdx.x * 32 + tx;
    unsigned long long mb = 0ull;
    if (j < n) {
        if (kkey)
            for (int64_t k = ty; k < K; k += 8) mb = max(mb, scaled_key(as_f64(src[k * lds + j]), key_exp(kkey[k])));
        else
            for (int64_t k = ty; k < K; k += 8) mb = max(mb, abs_bits(as_f64(src[k * lds + j])));
    }
    part[ty][tx] = mb;
    __syncthreads();
    if (ty == 0 && j < n) {
        for (int w = 1; w < 8; ++w) mb = max(mb, part[w][tx]);
        exps[j] = kkey ? key_exp(mb) : scale_exp(__longlong_as_double((long long)mb));
    }
}

// Column maximum keys of an m x K block (the inner-dimension scaling of the
// sliced Schur update): a CTA takes 32 columns and a strip of rows, its 8
// warps split the strip, and the strip's maximum goes to keys[k] by atomicMax
// (keys cleared before).
template <typename TS>
__global__ void k_col_keys(const TS *src, int64_t lds, int64_t m, int64_t K, unsigned long long *keys) {
    __shared__ unsigned long long part[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t k = (int64_t)blockIdx.x * 32 + tx;
    const int64_t rows = (m + gridDim.y - 1) / gridDim.y;
    const int64_t r0 = (int64_t)blockIdx.y * rows, r1 = r0 + rows < m ? r0 + rows : m;
    unsigned long long mb = 0ull;
    if (k < K)
        for (int64_t i = r0 + ty; i < r1; i += 8) mb = max(mb, scaled_key(as_f64(src[i * lds + k]), 0));
    part[ty][tx] = mb;
    __syncthreads();
    if (ty == 0 && k < K) {
        for (int w = 1; w < 8; ++w) mb = max(mb, part[w][tx]);
        if (mb) atomicMax(keys + k, mb);
    }
}

// Pass 2: 32 x 32 tiles through shared memory so both sides stay coalesced.
template <int ND, typename TS>
__global__ void k_slice_cols_T(const TS *src, int64_t lds, int64_t K, int64_t n, int64_t kpad,
                               __nv_bfloat16 *dst, int64_t ldq, const int *exps, const unsigned long long *kkey) {
    __shared__ double tile[32][33];
    const int64_t k0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        const int64_t k = k0 + r, j = j0 + tx;
        tile[r][tx] = (k < K && j < n) ? as_f64(src[k * lds + j]) : 0.0;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t j = j0 + r, k = k0 + tx;
        if (j < n && k < kpad) {
            float d[ND] = {};
            if (k < K) digits<ND>(tile[tx][r], exps[j], d, kkey ? key_exp(kkey[k]) : 0);
            put<ND>(dst + j * ldq, kpad, k, d);
        }
    }
}

// Both passes in one for a shallow operand (K <= 128, the inner blocks of
// the sliced factorization): a CTA holds its 32 columns whole in shared
// memory, takes their exponents, and slices them.
constexpr int kColsSmallK = 128;
template <int ND, typename TS>
__global__ void k_slice_cols_T_small(const TS *src, int64_t lds, int64_t K, int64_t n, int64_t kpad,
                                     __nv_bfloat16 *dst, int64_t ldq, int *exps, const unsigned long long *kkey) {
    __shared__ double tile[kColsSmallK][33];
    __shared__ unsigned long long part[8][33];
    __shared__ int ej[32];
    const int64_t j0 = (int64_t)blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    const int64_t j = j0 + tx;
    unsigned long long mb = 0ull;
    for (int k = ty; k < (int)K; k += 8) {
        const double x = j < n ? as_f64(src[k * lds + j]) : 0.0;
        tile[k][tx] = x;
        mb = max(mb, kkey ? scaled_key(x, key_exp(kkey[k])) : abs_bits(x));
    }
    part[ty][tx] = mb;
    __syncthreads();
    if (ty == 0) {
        for (int w = 1; w < 8; ++w) mb = max(mb, part[w][tx]);
        const int e = kkey ? key_exp(mb) : scale_exp(__longlong_as_double((long long)mb));
        ej[tx] = e;
        if (j < n) exps[j] = e;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t jr = j0 + r;
        if (jr >= n) break;
        for (int k = tx; k < (int)kpad; k += 32) {
            float d[ND] = {};
            if (k < K) digits<ND>(tile[k][r], ej[r], d, kkey ? key_exp(kkey[k]) : 0);
            put<ND>(dst + jr * ldq, kpad, k, d);
        }
    }
}

// Double-float <-> FP64 copies of a block (grid-stride over rows, coalesced columns).
// With amax, also max |src| into the status word *amax (the integer maximum
// of the magnitudes' bit patterns: a NaN outranks every number).
__global__ void k_df_from_f64(const double *src, int64_t lds, dfloat *dst, int64_t ldd, int64_t m, int64_t n,
                              unsigned long long *amax) {
    unsigned long long mb = 0ull;
    for (int64_t i = blockIdx.y; i < m; i += gridDim.y)
        for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
            const double v = src[i * lds + j];
            mb = max(mb, (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull);
            dst[i * ldd + j] = dfloat(v);
        }
    if (amax) {
        for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
        if ((threadIdx.x & 31) == 0 && mb) atomicMax(amax, mb);
    }
}
__global__ void k_df_to_f64(const dfloat *src, int64_t lds, double *dst, int64_t ldd, int64_t m, int64_t n) {
    for (int64_t i = blockIdx.y; i < m; i += gridDim.y)
        for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
            dst[i * ldd + j] = (double)src[i * lds + j];
}

__global__ void k_df_axpby(double alpha, const dfloat *W, int64_t ldw, double beta, double *D, int64_t ldd,
                           int64_t m, int64_t n) {
    for (int64_t i = blockIdx.y; i < m; i += gridDim.y)
        for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
            const dfloat w = W[i * ldw + j];
            const double v = alpha * (double)w.hi + alpha * (double)w.lo;
            D[i * ldd + j] = beta == 0.0 ? v : v + beta * D[i * ldd + j];
        }
}

// dst (m x n, FP64) = src^T (src n x m, double-float), 32 x 32 tiles through
// shared memory so reads and writes stay coalesced.
__global__ void k_df_to_f64_T(const dfloat *src, int64_t lds, double *dst, int64_t ldd, int64_t m, int64_t n) {
    __shared__ double tile[32][33];
    const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;   // dst rows i, columns j
    const int tx = threadIdx.x, ty = threadIdx.y;                                // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        const int64_t j = j0 + r, i = i0 + tx;                                    // src[j][i]
        tile[r][tx] = (j < n && i < m) ? (double)src[j * lds + i] : 0.0;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t i = i0 + r, j = j0 + tx;
        if (i < m && j < n) dst[i * ldd + j] = tile[tx][r];
    }
}

dim3 block_grid(int64_t m, int64_t n) {
    const int64_t gx = cdiv(n, 256) < 8 ? cdiv(n, 256) : 8;
    return dim3((unsigned)gx, (unsigned)(m < 65535 ? m : 65535));
}

}  // namespace

int64_t sliced_kpad(int64_t K) { return (K + 63) / 64 * 64; }
int sliced_slices(int nd) { return nd; }
int sliced_digits() { return g_default_digits; }
int set_sliced_digits(int nd) {
    if (!sliced::factor_supported(nd)) return -1;
    const int old = g_default_digits;
    g_default_digits = nd;
    return old;
}
int sliced_precond_digits() { return g_precond_digits; }
int sliced_mult_digits() { return g_mult_digits; }
int set_sliced_mult_digits(int d) {
    if (d != 1 && d != 2) return -1;
    const int old = g_mult_digits;
    g_mult_digits = d;
    return old;
}
int set_sliced_precond_digits(int nd) {
    if (!sliced::supported(nd)) return -1;
    const int old = g_precond_digits;
    g_precond_digits = nd;
    return old;
}

namespace {
template <typename TS>
cudaError_t slice_rows_t(int nd, const TS *src, int64_t lds, int64_t m, int64_t K, __nv_bfloat16 *dst, int64_t ldq,
                         int *exps, cudaStream_t s, const unsigned long long *kexp) {
    if (m <= 0) return cudaSuccess;
    if (nd < 1 || nd > 7 || ldq < nd * sliced_kpad(K)) return cudaErrorInvalidValue;
    int blocks = (int)((m + 7) / 8);
    if (blocks > 152 * 16) blocks = 152 * 16;
    const int64_t kpad = sliced_kpad(K);
    note_launch();
    switch (nd) {
        case 1: k_slice_rows<1, TS><<<blocks, 256, 0, s>>>(src, lds, m, K, kpad, dst, ldq, exps, kexp); break;
        case 2: k_slice_rows<2, TS><<<blocks, 256, 0, s>>>(src, lds, m, K, kpad, dst, ldq, exps, kexp); break;
        case 3: k_slice_rows<3, TS><<<blocks, 256, 0, s>>>(src, lds, m, K, kpad, dst, ldq, exps, kexp); break;
        case 4: k_slice_rows<4, TS><<<blocks, 256, 0, s>>>(src, lds, m, K, kpad, dst, ldq, exps, kexp); break;
        case 5: k_slice_rows<5, TS><<<blocks, 256, 0, s>>>(src, lds, m, K, kpad, dst, ldq, exps, kexp); break;
        case 6: k_slice_rows<6, TS><<<blocks, 256, 0, s>>>(src, lds, m, K, kpad, dst, ldq, exps, kexp); break;
        default: k_slice_rows<7, TS><<<blocks, 256, 0, s>>>(src, lds, m, K, kpad, dst, ldq, exps, kexp); break;
    }
    return cudaGetLastError();
}

template <typename TS>
cudaError_t slice_cols_T_t(int nd, const TS *src, int64_t lds, int64_t K, int64_t n, __nv_bfloat16 *dst,
                           int64_t ldq, int *exps, cudaStream_t s, const unsigned long long *kexp) {
    if (n <= 0) return cudaSuccess;
    const int64_t kpad = sliced_kpad(K);
    if (nd < 1 || nd > 7 || ldq < nd * kpad) return cudaErrorInvalidValue;
    if (kpad <= kColsSmallK) {
        const unsigned gx = (unsigned)cdiv(n, 32);
        note_launch();
        switch (nd) {
            case 1: k_slice_cols_T_small<1, TS><<<gx, dim3(32, 8), 0, s>>>(src, lds, K, n, kpad, dst, ldq, exps, kexp); break;
            case 2: k_slice_cols_T_small<2, TS><<<gx, dim3(32, 8), 0, s>>>(src, lds, K, n, kpad, dst, ldq, exps, kexp); break;
            case 3: k_slice_cols_T_small<3, TS><<<gx, dim3(32, 8), 0, s>>>(src, lds, K, n, kpad, dst, ldq, exps, kexp); break;
            case 4: k_slice_cols_T_small<4, TS><<<gx, dim3(32, 8), 0, s>>>(src, lds, K, n, kpad, dst, ldq, exps, kexp); break;
            case 5: k_slice_cols_T_small<5, TS><<<gx, dim3(32, 8), 0, s>>>(src, lds, K, n, kpad, dst, ldq, exps, kexp); break;
            case 6: k_slice_cols_T_small<6, TS><<<gx, dim3(32, 8), 0, s>>>(src, lds, K, n, kpad, dst, ldq, exps, kexp); break;
            default: k_slice_cols_T_small<7, TS><<<gx, dim3(32, 8), 0, s>>>(src, lds, K, n, kpad, dst, ldq, exps, kexp); break;
        }
        return cudaGetLastError();
    }
    note_launch();
    k_col_exps<TS><<<(unsigned)cdiv(n, 32), 256, 0, s>>>(src, lds, K, n, exps, kexp);
    dim3 g((unsigned)cdiv(n, 32), (unsigned)cdiv(kpad, 32));
    if (g.y > 65535u) return cudaErrorInvalidValue;
    note_launch();
    switch (nd) {
        case 1: k_slice_cols_T<1, TS><<<g, dim3(32, 8), 0, s>>>(src, lds, K, n, kpad, dst, ldq, exps, kexp); break;
        case 2: k_slice_cols_T<2, TS><<<g, dim3(32, 8), 0, s>>>(src, lds, K, n, kpad, dst, ldq, exps, kexp); break;
        case 3: k_slice_cols_T<3, TS><<<g, dim3(32, 8), 0, s>>>(src, lds, K, n, kpad, dst, ldq, exps, kexp); break;
        case 4: k_slice_cols_T<4, TS><<<g, dim3(32, 8), 0, s>>>(src, lds, K, n, kpad, dst, ldq, exps, kexp); break;
        case 5: k_slice_cols_T<5, TS><<<g, dim3(32, 8), 0, s>>>(src, lds, K, n, kpad, dst, ldq, exps, kexp); break;
        case 6: k_slice_cols_T<6, TS><<<g, dim3(32, 8), 0, s>>>(src, lds, K, n, kpad, dst, ldq, exps, kexp); break;
        default: k_slice_cols_T<7, TS><<<g, dim3(32, 8), 0, s>>>(src, lds, K, n, kpad, dst, ldq, exps, kexp); break;
    }
    return cudaGetLastError();
}

template <typename TS>
cudaError_t sliced_inner_exps_t(const TS *L, int64_t ldl, int64_t m, int64_t K, unsigned long long *keys,
                                cudaStream_t s) {
    if (K <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(keys, 0, (size_t)K * sizeof(unsigned long long), s);
    if (e != cudaSuccess || m <= 0) return e;
    // about two CTAs per SM over the strips
    const int64_t gx = cdiv(K, 32);
    int64_t gy = (152 * 2 + gx - 1) / gx;
    gy = gy < cdiv(m, 64) ? gy : cdiv(m, 64);
    note_launch();
    k_col_keys<TS><<<dim3((unsigned)gx, (unsigned)(gy > 0 ? gy : 1)), 256, 0, s>>>(L, ldl, m, K, keys);
    return cudaGetLastError();
}
}  // namespace

cudaError_t slice_rows(int nd, const double *src, int64_t lds, int64_t m, int64_t K, __nv_bfloat16 *dst, int64_t ldq,
                       int *exps, cudaStream_t s, const unsigned long long *kexp) {
    return slice_rows_t(nd, src, lds, m, K, dst, ldq, exps, s, kexp);
}
cudaError_t slice_rows(int nd, const dfloat *src, int64_t lds, int64_t m, int64_t K, __nv_bfloat16 *dst, int64_t ldq,
                       int *exps, cudaStream_t s, const unsigned long long *kexp) {
    return slice_rows_t(nd, src, lds, m, K, dst, ldq, exps, s, kexp);
}
cudaError_t slice_cols_T(int nd, const double *src, int64_t lds, int64_t K, int64_t n, __nv_bfloat16 *dst,
                         int64_t ldq, int *exps, cudaStream_t s, const unsigned long long *kexp) {
    return slice_cols_T_t(nd, src, lds, K, n, dst, ldq, exps, s, kexp);
}
cudaError_t slice_cols_T(int nd, const dfloat *src, int64_t lds, int64_t K, int64_t n, __nv_bfloat16 *dst,
                         int64_t ldq, int *exps, cudaStream_t s, const unsigned long long *kexp) {
    return slice_cols_T_t(nd, src, lds, K, n, dst, ldq, exps, s, kexp);
}
cudaError_t sliced_inner_exps(const double *L, int64_t ldl, int64_t m, int64_t K, unsigned long long *keys,
                              cudaStream_t s) {
    return sliced_inner_exps_t(L, ldl, m, K, keys, s);
}
cudaError_t sliced_inner_exps(const dfloat *L, int64_t ldl, int64_t m, int64_t K, unsigned long long *keys,
                              cudaStream_t s) {
    return sliced_inner_exps_t(L, ldl, m, K, keys, s);
}

cudaError_t df_from_f64(const double *src, int64_t lds, dfloat *dst, int64_t ldd, int64_t m, int64_t n,
                        cudaStream_t s, unsigned long long *amax) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    note_launch();
    k_df_from_f64<<<block_grid(m, n), 256, 0, s>>>(src, lds, dst, ldd, m, n, amax);
    return cudaGetLastError();
}

cudaError_t df_to_f64(const dfloat *src, int64_t lds, double *dst, int64_t ldd, int64_t m, int64_t n,
                      cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    note_launch();
    k_df_to_f64<<<block_grid(m, n), 256, 0, s>>>(src, lds, dst, ldd, m, n);
    return cudaGetLastError();
}

cudaError_t df_to_f64_T(const dfloat *src, int64_t lds, double *dst, int64_t ldd, int64_t m, int64_t n,
                        cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    dim3 g((unsigned)cdiv(n, 32), (unsigned)cdiv(m, 32));
    if (g.y > 65535u) return cudaErrorInvalidValue;
    note_launch();
    k_df_to_f64_T<<<g, dim3(32, 8), 0, s>>>(src, lds, dst, ldd, m, n);
    return cudaGetLastError();
}

cudaError_t df_axpby(double alpha, const dfloat *W, int64_t ldw, double beta, double *D, int64_t ldd, int64_t m,
                     int64_t n, cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    note_launch();
    k_df_axpby<<<block_grid(m, n), 256, 0, s>>>(alpha, W, ldw, beta, D, ldd, m, n);
    return cudaGetLastError();
}

cudaError_t sliced_matmul(int nd, int64_t m, int64_t n, int64_t K, const double *A, int64_t lda, const double *B,
                          int64_t ldb, dfloat *D, int64_t ldd, __nv_bfloat16 *Aq, __nv_bfloat16 *Bq, int *exps,
                          cudaStream_t s, int ndb) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    const int nda = nd;
    if (ndb <= 0) ndb = nd;
    cudaError_t e = cudaMemset2DAsync(D, (size_t)ldd * sizeof(dfloat), 0, (size_t)n * sizeof(dfloat), (size_t)m, s);
    const int64_t chunk = nda <= 2 ? kSlicedChunk2 : kSlicedChunk;
    for (int64_t k0 = 0; k0 < K && e == cudaSuccess; k0 += chunk) {
        const int64_t kc = K - k0 < chunk ? K - k0 : chunk;
        const int64_t kpad = sliced_kpad(kc), lda_q = nda * kpad, ldb_q = ndb * kpad;
        e = slice_rows(nda, A + k0, lda, m, kc, Aq, lda_q, exps, s);
        if (e == cudaSuccess) e = slice_cols_T(ndb, B + k0 * ldb, ldb, kc, n, Bq, ldb_q, exps + m, s);
        if (e == cudaSuccess)
            e = tc_gemm_sliced2(nda, ndb, m, n, kpad, 1.0f, Aq, lda_q, Bq, ldb_q, exps, exps + m, D, ldd, s);
    }
    return e;
}

cudaError_t sliced_matmul_t(int nda, int ndb, int64_t m, int64_t n, int64_t K, const double *A, int64_t lda,
                            const double *B, int64_t ldb, dfloat *Dt, int64_t lddt, __nv_bfloat16 *Bq,
                            __nv_bfloat16 *Aq, int *exps, cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemset2DAsync(Dt, (size_t)lddt * sizeof(dfloat), 0, (size_t)m * sizeof(dfloat), (size_t)n, s);
    const int64_t chunk = ndb <= 2 ? kSlicedChunk2 : kSlicedChunk;
    for (int64_t k0 = 0; k0 < K && e == cudaSuccess; k0 += chunk) {
        const int64_t kc = K - k0 < chunk ? K - k0 : chunk;
        const int64_t kpad = sliced_kpad(kc), ldq_b = ndb * kpad, ldq_a = nda * kpad;
        // M side: the columns of B (ndb digits); N side: the rows of A (nda digits)
        e = slice_cols_T(ndb, B + k0 * ldb, ldb, kc, n, Bq, ldq_b, exps, s);
        if (e == cudaSuccess) e = slice_rows(nda, A + k0, lda, m, kc, Aq, ldq_a, exps + n, s);
        if (e == cudaSuccess)
            e = tc_gemm_sliced2(ndb, nda, n, m, kpad, 1.0f, Bq, ldq_b, Aq, ldq_a, exps, exps + n, Dt, lddt, s);
    }
    return e;
}

}  // namespace genp
