// rng.cu -- random multipliers from a counter-based generator.
//
// Generator: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 3.3):
// ten rounds, each taking the 128-bit products of words 0 and 2 with two
// fixed odd multipliers, xoring the high halves into words 1 and 3 with the
// round key, and bumping the key by two Weyl increments between rounds.
// Layout of the method's draws: key = (seed, stream_id); counter =
// (index, block, tag, t).  Gaussian entries use Marsaglia's polar method
// with a logarithm built from IEEE basic operations only (the atanh series
// of ln((1+f)/(1-f)), Abramowitz & Stegun 4.1.27), so that every entry is
// reproducible bit for bit on any IEEE machine.  The _rn intrinsics below
// keep the compiler from fusing multiply-adds in this file.
#include "genp_internal.cuh"

#include "e4m3.cuh"

namespace genp {
namespace {

constexpr uint64_t kTagDense = 0x10, kTagCirc = 0x11, kTagPerm = 0x12, kTagSign = 0x13;
constexpr int kPolarBlocks = 32;

struct U4 { uint64_t w[4]; };

__device__ __forceinline__ U4 philox(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0,
                                     uint64_t k1) {
    const uint64_t m0 = 0xD2E7470EE14C6C93ull, m1 = 0xCA5A826395121157ull;
    const uint64_t w0 = 0x9E3779B97F4A7C15ull, w1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += w0; k1 += w1; }
        const uint64_t hi0 = __umul64hi(m0, c0), lo0 = m0 * c0;
        const uint64_t hi1 = __umul64hi(m1, c2), lo1 = m1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    U4 o;
    o.w[0] = c0; o.w[1] = c1; o.w[2] = c2; o.w[3] = c3;
    return o;
}

__device__ __forceinline__ double unit53(uint64_t w) {
    return __dmul_rn((double)(w >> 11), 1.1102230246251565e-16 /* 2^-53 */);
}

// ln(s) for positive normal s: s = m 2^e exactly, m in (sqrt2/2, sqrt2],
// ln m = 2 atanh(f), f = (m-1)/(m+1), |f| < 0.172, series to f^23.
__device__ double ln_series(double s) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(s);
    int e = (int)((b >> 52) & 0x7ffull) - 1023;
    double m = __longlong_as_double((long long)((b & 0x000FFFFFFFFFFFFFull) | (1023ull << 52)));
    if (m > 1.4142135623730951) { m = __dmul_rn(m, 0.5); e += 1; }
    const double f = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
    const double f2 = __dmul_rn(f, f);
    // 1/(2k+1), k = 0..11, each the correctly rounded double (what IEEE
    // division 1.0 / (2k+1) gives), as constants instead of 12 divisions
    constexpr double kInvOdd[12] = {0x1.0000000000000p+0, 0x1.5555555555555p-2, 0x1.999999999999ap-3,
                                    0x1.2492492492492p-3, 0x1.c71c71c71c71cp-4, 0x1.745d1745d1746p-4,
                                    0x1.3b13b13b13b14p-4, 0x1.1111111111111p-4, 0x1.e1e1e1e1e1e1ep-5,
                                    0x1.af286bca1af28p-5, 0x1.8618618618618p-5, 0x1.642c8590b2164p-5};
    const int K = 11;
    double p = kInvOdd[K];
#pragma unroll
    for (int k = K - 1; k >= 0; --k) p = __dadd_rn(__dmul_rn(p, f2), kInvOdd[k]);
    const double lm = __dmul_rn(__dmul_rn(2.0, f), p);
    const double el = __dmul_rn((double)e, 0.6931471805599453);
    return __dadd_rn(el, lm);
}

// The accepted pair is searched first (cheap, divergent), the logarithm,
// division and square root are then taken once per warp with every lane
// converged: lanes that accept at different tries would otherwise run the
// expensive part once per try position.
__device__ double polar_normal(uint64_t seed, uint64_t sid, uint64_t tag, uint64_t idx) {
    double v1 = 0.0, s = 0.0;
    bool found = false;
    for (uint64_t blk = 0; blk < kPolarBlocks && !found; ++blk) {
        const U4 w = philox(idx, blk, tag, 0, seed, sid);
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const double a = __dsub_rn(__dmul_rn(2.0, unit53(w.w[2 * p])), 1.0);
            const double b = __dsub_rn(__dmul_rn(2.0, unit53(w.w[2 * p + 1])), 1.0);
            const double q = __dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b));
            if (!found && q > 0.0 && q < 1.0) {
                v1 = a;
                s = q;
                found = true;
            }
        }
    }
    if (!found) return 0.0;
    double t = ln_series(s);
    t = __dmul_rn(-2.0, t);
    t = __ddiv_rn(t, s);
    t = __dsqrt_rn(t);
    return __dmul_rn(v1, t);
}

// The same polar method in IEEE single precision (multipliers on the FP32
// grid): 24-bit uniforms, atanh series to f^11, tags shifted by 4.
__device__ float ln_series_f32(float s) {
    const unsigned b = __float_as_uint(s);
    int e = (int)((b >> 23) & 0xffu) - 127;
    float m = __uint_as_float((b & 0x007FFFFFu) | (127u << 23));
    if (m > 1.41421354f) { m = __fmul_rn(m, 0.5f); e += 1; }
    const float f = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float f2 = __fmul_rn(f, f);
    // 1/(2k+1), k = 0..5, correctly rounded to single precision
    constexpr float kInvOddF[6] = {0x1.000000p+0f, 0x1.555556p-2f, 0x1.99999ap-3f,
                                   0x1.24924ap-3f, 0x1.c71c72p-4f, 0x1.745d18p-4f};
    const int K = 5;
    float p = kInvOddF[K];
#pragma unroll
    for (int k = K - 1; k >= 0; --k) p = __fadd_rn(__fmul_rn(p, f2), kInvOddF[k]);
    const float lm = __fmul_rn(__fmul_rn(2.0f, f), p);
    const float el = __fmul_rn((float)e, 0.693147182f);
    return __fadd_rn(el, lm);
}

__device__ float polar_normal_f32(uint64_t seed, uint64_t sid, uint64_t tag, uint64_t idx) {
    float v1 = 0.0f, s = 0.0f;
    bool found = false;
    for (uint64_t blk = 0; blk < kPolarBlocks && !found; ++blk) {
        const U4 w = philox(idx, blk, tag, 0, seed, sid);
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const float u1 = __fmul_rn((float)(uint32_t)(w.w[2 * p] >> 40), 5.96046448e-8f /* 2^-24 */);
            const float u2 = __fmul_rn((float)(uint32_t)(w.w[2 * p + 1] >> 40), 5.96046448e-8f);
            const float a = __fsub_rn(__fmul_rn(2.0f, u1), 1.0f);
            const float b = __fsub_rn(__fmul_rn(2.0f, u2), 1.0f);
            const float q = __fadd_rn(__fmul_rn(a, a), __fmul_rn(b, b));
            if (!found && q > 0.0f && q < 1.0f) {
                v1 = a;
                s = q;
                found = true;
            }
        }
    }
    if (!found) return 0.0f;
    float t = ln_series_f32(s);
    t = __fmul_rn(-2.0f, t);
    t = __fdiv_rn(t, s);
    t = __fsqrt_rn(t);
    return __fmul_rn(v1, t);
}

// Round a finite double to the nearest BF16 value (ties to even) by clearing
// the 45 low mantissa bits with a round-to-nearest-even bias.
__device__ __forceinline__ double round_to_bf16_grid(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long lsb = (b >> 45) & 1ull;
    b += 0x00000FFFFFFFFFFFull + lsb;
    b &= ~0x00001FFFFFFFFFFFull;
    return __longlong_as_double((long long)b);
}

// FP8 grid: e4m3 values times 2^e, one e for the matrix: the least integer
// with 12.5 scale <= 448 2^e (12.5 standard deviations bound every polar
// draw), so no entry saturates.  Rounding to nearest, ties to even.
__host__ __device__ inline int fp8_grid_exp(double scale) {
    const double amax = 12.5 * scale;
    if (!(amax > 0.0)) return 0;
    int p = 0;
    const double f = frexp(amax, &p);
    const int e = f <= 0.875 ? p - 9 : p - 8;
    return e < -126 ? -126 : (e > 126 ? 126 : e);
}
__device__ __forceinline__ double round_to_fp8_grid(double v, int e) {
    // the scalings by 2^-e and 2^e are exact (|e| <= 126)
    const double down = __longlong_as_double((long long)(1023 - e) << 52);
    const double up = __longlong_as_double((long long)(1023 + e) << 52);
    return e4m3_round_f64(v * down) * up;
}

// Fixed-point grid of the sliced product: integer multiples of 2^(E - 13)
// with E the least integer such that 12.5 scale <= 2^E (12.5 standard
// deviations bound every polar draw), so |entry| < 2^E holds 14 signed bits
// at any column scale 2^f <= 2^E: two exact balanced base-128 digits.  The
// one-digit grid (the dense Gaussian's, by genp_sliced_multiplier_digits):
// multiples of 2^(E - 6), one exact digit.  qb below is 13 or 6.
// Rounding to nearest, ties to even.
__host__ __device__ inline int sliced_grid_exp(double scale) {
    const double amax = 12.5 * scale;
    if (!(amax > 0.0)) return 0;
    int p = 0;
    const double f = frexp(amax, &p);    // amax = f 2^p, f in [0.5, 1)
    const int e = f == 0.5 ? p - 1 : p;
    return e < -1000 ? -1000 : (e > 1000 ? 1000 : e);
}
__device__ __forceinline__ double round_to_sliced_grid(double v, int e, int qb = 13) {
    // v 2^(qb - e) and back: exact power-of-two scalings (|e| <= 1000)
    const double down = __longlong_as_double((long long)(1023 + qb - e) << 52);
    const double up = __longlong_as_double((long long)(1023 - qb + e) << 52);
    return rint(v * down) * up;
}

// The same rounding of an FP32 draw v (|v| < 2^e by the 12.5-deviation
// bound), all in FP32: v 2^(13 - e) has at most 24 significant bits and
// magnitude below 2^13, so rintf (ties to even) and both power-of-two
// scalings are exact and give the FP64 rounding's value bit for bit, without
// FP64 operations (a sixty-fourth of the FP32 rate on this GPU).
__device__ __forceinline__ double round_to_sliced_grid_f32(float v, int e, int qb = 13) {
    const float down = __uint_as_float((uint32_t)(127 + qb - e) << 23);
    const float up = __uint_as_float((uint32_t)(127 - qb + e) << 23);
    return (double)__fmul_rn(rintf(__fmul_rn(v, down)), up);
}

__device__ __forceinline__ double on_grid(double v, genp_prec grid) {
    if (grid == GENP_BF16) return round_to_bf16_grid(v);
    if (grid == GENP_FP32) return (double)__double2float_rn(v);
    return v;
}

// One Gaussian entry of scale `scale` on the requested grid.  The FP32, FP8
// and sliced grids draw by the polar method in FP32 on their own tag (tag +
// 4); the FP8 grid then rounds that draw to e4m3 times 2^e and the sliced grid
// to a multiple of 2^(E - 13) (the draw's 24 bits are far beyond either).
// The FP64 and BF16 grids draw in FP64.
__device__ __forceinline__ double draw_on_grid(uint64_t seed, uint64_t sid, uint64_t tag, uint64_t idx, double scale,
                                               genp_prec grid) {
    if (grid == GENP_FP32 || grid == GENP_FP8_E4M3 || grid == GENP_BF16_SLICED) {
        const double v = (double)__fmul_rn(polar_normal_f32(seed, sid, tag + 4, idx), __double2float_rn(scale));
        if (grid == GENP_FP32) return v;
        return grid == GENP_FP8_E4M3 ? round_to_fp8_grid(v, fp8_grid_exp(scale))
                                     : round_to_sliced_grid(v, sliced_grid_exp(scale));
    }
    return on_grid(__dmul_rn(polar_normal(seed, sid, tag, idx), scale), grid);
}

__global__ void k_dense(double *G, int64_t n, uint64_t seed, uint64_t sid, double scale, genp_prec grid,
                        float *G32, __nv_bfloat16 *Gbf, int qb) {
    const int64_t total = n * n;
    // the sliced grid's exponent and the FP32 scale, once; the FP32 rounding
    // needs both scalings' exponents in the normal range
    const int ge = sliced_grid_exp(scale);
    const float sf = __double2float_rn(scale);
    const bool sliced_f32_ok = ge > -100 && ge < 100;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const double v = grid == GENP_BF16_SLICED && sliced_f32_ok
                             ? round_to_sliced_grid_f32(__fmul_rn(polar_normal_f32(seed, sid, kTagDense + 4, (uint64_t)idx), sf),
                                                        ge, qb)
                             : grid == GENP_BF16_SLICED
                                   ? round_to_sliced_grid((double)__fmul_rn(polar_normal_f32(seed, sid, kTagDense + 4,
                                                                                             (uint64_t)idx),
                                                                            sf),
                                                          ge, qb)
                                   : draw_on_grid(seed, sid, kTagDense, (uint64_t)idx, scale, grid);
        G[idx] = v;
        if (G32) G32[idx] = (float)v;
        if (Gbf) Gbf[(idx % n) * round8(n) + idx / n] = __float2bfloat16_rn((float)v);  // G^T, K-major
    }
}

__global__ void k_circ(double *g, int64_t n, uint64_t seed, uint64_t sid, double scale, genp_prec grid) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        g[i] = draw_on_grid(seed, sid, kTagCirc, (uint64_t)i, scale, grid);
}

// Gaussian Toeplitz multiplier (Definition 3.2): the 2n - 1 entries
// t_d (d = i - j in [-(n-1), n-1]) drawn at index d + n - 1 on their own tag,
// stored as the first column of the circulant of order 2n that embeds the
// Toeplitz matrix in its leading n x n block: g[d mod 2n] = t_d, g[n] = 0.
constexpr uint64_t kTagToep = 0x17, kTagHouse = 0x18;
__global__ void k_toeplitz(double *g, int64_t n, uint64_t seed, uint64_t sid, double scale, genp_prec grid) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < 2 * n; q += (int64_t)gridDim.x * blockDim.x) {
        if (q == 2 * n - 1) {
            g[n] = 0.0;
            continue;
        }
        const int64_t d = q - (n - 1);
        const double v = draw_on_grid(seed, sid, kTagToep, (uint64_t)q, scale, grid);
        g[d >= 0 ? d : 2 * n + d] = v;
    }
}

// Householder reflector I - 2 u u^T / n (the Householder multipliers of the
// tests Sec. 7.1 cites, read as an orthogonal reflector): u_i = +-1 from the
// low bit of Philox word 0 at (i, 0, tag, 0).
__global__ void k_householder(double *u, int64_t n, uint64_t seed, uint64_t sid) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const U4 w = philox((uint64_t)i, 0, kTagHouse, 0, seed, sid);
        u[i] = (w.w[0] & 1ull) ? -1.0 : 1.0;
    }
}

// The m x r sketch of the low-rank approximation (Proto-Alg. 5.1, Stage 1;
// Sec. 7.2): Gaussian G[i][j] = scale z(i r + j), or Gaussian Toeplitz
// G[i][j] = scale z(i - j + r - 1) (m + r - 1 independent draws).
constexpr uint64_t kTagSketch = 0x19, kTagSketchToep = 0x1A;
__global__ void k_sketch(double *G, int64_t ldg, int64_t m, int64_t r, int toeplitz, uint64_t seed, uint64_t sid,
                         double scale) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m * r; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q / r, j = q % r;
        const double z = toeplitz ? polar_normal(seed, sid, kTagSketchToep, (uint64_t)(i - j + r - 1))
                                  : polar_normal(seed, sid, kTagSketch, (uint64_t)q);
        G[i * ldg + j] = __dmul_rn(z, scale);
    }
}

// Circulant with a +-1 first column (the paper's test multipliers): attempt
// a takes g_i from the low bit of Philox word 0 at (i, 0, tag, a) and is
// kept when no DFT bin of power-of-two order vanishes.  Exact integer test:
// the bin at frequency 0 is sum g_i; the bins at the primitive 2m-th roots of
// unity (2m | n) all vanish iff every folded sum h_r = sum_q (-1)^q g_{r+qm}
// (r < m) is zero, x^m + 1 being irreducible over the rationals.  One CTA.
constexpr uint64_t kTagCircPm1 = 0x16;
__global__ void k_circ_pm1(double *g, int64_t n, uint64_t seed, uint64_t sid, int *attempt) {
    __shared__ unsigned long long acc;
    __shared__ int reject;
    int a = 0;
    for (; a < 64; ++a) {
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            const U4 w = philox((uint64_t)i, 0, kTagCircPm1, (uint64_t)a, seed, sid);
            g[i] = (w.w[0] & 1ull) ? -1.0 : 1.0;
        }
        if (threadIdx.x == 0) {
            acc = 0ull;
            reject = 0;
        }
        __syncthreads();
        long long dc = 0;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) dc += (long long)g[i];
        atomicAdd(&acc, (unsigned long long)dc);
        __syncthreads();
        if (threadIdx.x == 0 && (long long)acc == 0) reject = 1;
        __syncthreads();
        for (int64_t m = 1; !reject && 2 * m <= n && n % (2 * m) == 0; m *= 2) {
            if (threadIdx.x == 0) acc = 0ull;
            __syncthreads();
            int nonzero = 0;
            for (int64_t r = threadIdx.x; r < m && !nonzero; r += blockDim.x) {
                long long h = 0;
                for (int64_t q = 0; q < n / m; ++q) h += ((q & 1) ? -1 : 1) * (long long)g[r + q * m];
                if (h != 0) nonzero = 1;
            }
            if (nonzero) atomicOr(&acc, 1ull);
            __syncthreads();
            if (threadIdx.x == 0 && acc == 0ull) reject = 1;
            __syncthreads();
        }
        const int rej = reject;
        __syncthreads();
        if (!rej) break;
    }
    if (threadIdx.x == 0) *attempt = a;
}

// Uniform integer in [0, range) (Lemire's multiply-shift with rejection).
__device__ uint64_t bounded(uint64_t range, uint64_t seed, uint64_t sid, uint64_t i, uint64_t t) {
    const uint64_t thr = (0ull - range) % range;
    uint64_t hi = 0;
    for (uint64_t blk = 0; blk < 16; ++blk) {
        const U4 w = philox(i, blk, kTagPerm, t, seed, sid);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            hi = __umul64hi(w.w[q], range);
            const uint64_t lo = w.w[q] * range;
            if (lo >= thr) return hi;
        }
    }
    return hi;
}

// Draws of the Fisher-Yates shuffle: swap partner of position i (i >= 1) and the signs.
__global__ void k_perm_draws(int32_t *draws, int8_t *signs, int64_t n, int nnz, uint64_t seed, uint64_t sid) {
    const int64_t total = n * nnz;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = idx / n, i = idx % n;
        draws[idx] = i >= 1 ? (int32_t)bounded((uint64_t)(i + 1), seed, sid, (uint64_t)i, (uint64_t)t) : 0;
        const U4 w = philox((uint64_t)i, 0, kTagSign, (uint64_t)t, seed, sid);
        signs[idx] = (w.w[0] & 1ull) ? (int8_t)-1 : (int8_t)1;
    }
}

// The shuffle itself is sequential: one thread per permutation, i = n-1 .. 1.
__global__ void k_perm_shuffle(int32_t *rows, const int32_t *draws, int64_t n) {
    if (threadIdx.x != 0) return;
    const int64_t t = blockIdx.x;
    int32_t *p = rows + t * n;
    const int32_t *d = draws + t * n;
    for (int64_t i = n - 1; i >= 1; --i) {
        const int64_t j = d[i];
        const int32_t tmp = p[i];
        p[i] = p[j];
        p[j] = tmp;
    }
}

__global__ void k_iota(int32_t *rows, int64_t n, int nnz) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * nnz;
         idx += (int64_t)gridDim.x * blockDim.x)
        rows[idx] = (int32_t)(idx % n);
}

__global__ void k_invert(const int32_t *rows, const int8_t *signs, int32_t *inv_rows, int8_t *inv_signs,
                         int64_t n, int nnz) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * nnz;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = idx / n, j = idx % n;
        const int64_t r = rows[idx];
        inv_rows[t * n + r] = (int32_t)j;
        inv_signs[t * n + r] = signs[idx];
    }
}

__global__ void k_circ_dense(const double *g, int64_t cn, int64_t n, double *G, int64_t ldg) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / n, j = idx % n;
        int64_t d = i - j;
        if (d < 0) d += cn;
        G[i * ldg + j] = g[d];
    }
}

__global__ void k_zero(double *G, int64_t n, int64_t ldg) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * n;
         idx += (int64_t)gridDim.x * blockDim.x)
        G[(idx / n) * ldg + idx % n] = 0.0;
}

// One thread per column: entries of one column never race.
__global__ void k_sparse_dense(const int32_t *rows, const int8_t *signs, int64_t n, int nnz, double *G,
                               int64_t ldg) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        for (int t = 0; t < nnz; ++t) {
            const int64_t r = rows[(int64_t)t * n + j];
            G[r * ldg + j] += (double)signs[(int64_t)t * n + j];
        }
}

// Multipliers of a batch, drawn in single precision (FP32 grid): system i's
// dense G (n x n, at mat_off) or circulant first column g (n, at g_off) with
// stream id sid_i, entries scale_i * z32(idx), scale_i = fl32(1/sqrt(n_i))
// for the dense kind and 1 for the circulant.  One CTA per system.
__global__ void k_batch_draw(const BatchDesc *d, int count, uint64_t seed, int circ, float *Gpool, float *gpool) {
    for (int s = blockIdx.x; s < count; s += gridDim.x) {
        const BatchDesc q = d[s];
        if (circ) {
            for (int64_t i = threadIdx.x; i < q.n; i += blockDim.x)
                gpool[q.g_off + i] = polar_normal_f32(seed, (uint64_t)q.sid, kTagCirc + 4, (uint64_t)i);
        } else {
            const float scale = __double2float_rn(1.0 / sqrt((double)q.n));
            for (int64_t idx = threadIdx.x; idx < q.n * q.n; idx += blockDim.x)
                Gpool[q.mat_off + idx] =
                    __fmul_rn(polar_normal_f32(seed, (uint64_t)q.sid, kTagDense + 4, (uint64_t)idx), scale);
        }
    }
}

int grid_for(int64_t work, int threads) {
    int64_t b = cdiv(work, threads);
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

cudaError_t launch_make_dense(double *G, int64_t n, uint64_t seed, uint64_t sid, double scale, genp_prec grid,
                              float *G32, __nv_bfloat16 *Gbf, cudaStream_t s, int grid_digits) {
    if (grid_digits != 1 && grid_digits != 2) return cudaErrorInvalidValue;
    note_launch();
    k_dense<<<grid_for(n * n, 256), 256, 0, s>>>(G, n, seed, sid, scale, grid, G32, Gbf, 7 * grid_digits - 1);
    return cudaGetLastError();
}

cudaError_t launch_make_circulant(double *g, int64_t n, uint64_t seed, uint64_t sid, double scale,
                                  genp_prec grid, cudaStream_t s) {
    note_launch();
    k_circ<<<grid_for(n, 256), 256, 0, s>>>(g, n, seed, sid, scale, grid);
    return cudaGetLastError();
}

cudaError_t launch_make_toeplitz(double *g, int64_t n, uint64_t seed, uint64_t sid, double scale, genp_prec grid,
                                 cudaStream_t s) {
    note_launch();
    k_toeplitz<<<grid_for(2 * n, 256), 256, 0, s>>>(g, n, seed, sid, scale, grid);
    return cudaGetLastError();
}

cudaError_t launch_sketch(double *G, int64_t ldg, int64_t m, int64_t r, bool toeplitz, uint64_t seed, uint64_t sid,
                          double scale, cudaStream_t s) {
    note_launch();
    k_sketch<<<grid_for(m * r, 256), 256, 0, s>>>(G, ldg, m, r, toeplitz ? 1 : 0, seed, sid, scale);
    return cudaGetLastError();
}

cudaError_t launch_make_householder(double *u, int64_t n, uint64_t seed, uint64_t sid, cudaStream_t s) {
    note_launch();
    k_householder<<<grid_for(n, 256), 256, 0, s>>>(u, n, seed, sid);
    return cudaGetLastError();
}

cudaError_t launch_make_circulant_pm1(double *g, int64_t n, uint64_t seed, uint64_t sid, int *attempt,
                                      cudaStream_t s) {
    note_launch();
    k_circ_pm1<<<1, 1024, 0, s>>>(g, n, seed, sid, attempt);
    return cudaGetLastError();
}

cudaError_t launch_make_sparse(int32_t *rows, int8_t *signs, int32_t *inv_rows, int8_t *inv_signs,
                               int32_t *scratch, int64_t n, int nnz, uint64_t seed, uint64_t sid,
                               cudaStream_t s) {
    note_launch();
    k_perm_draws<<<grid_for(n * nnz, 256), 256, 0, s>>>(scratch, signs, n, nnz, seed, sid);
    note_launch();
    k_iota<<<grid_for(n * nnz, 256), 256, 0, s>>>(rows, n, nnz);
    note_launch();
    k_perm_shuffle<<<nnz, 32, 0, s>>>(rows, scratch, n);
    note_launch();
    k_invert<<<grid_for(n * nnz, 256), 256, 0, s>>>(rows, signs, inv_rows, inv_signs, n, nnz);
    return cudaGetLastError();
}

cudaError_t launch_batch_draw(const BatchDesc *d, int count, uint64_t seed, bool circ, float *Gpool, float *gpool,
                              cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    note_launch();
    k_batch_draw<<<152 * 8 < count ? 152 * 8 : count, 256, 0, s>>>(d, count, seed, circ ? 1 : 0, Gpool, gpool);
    return cudaGetLastError();
}

cudaError_t launch_circulant_to_dense(const double *g, int64_t cn, int64_t n, double *G, int64_t ldg,
                                      cudaStream_t s) {
    note_launch();
    k_circ_dense<<<grid_for(n * n, 256), 256, 0, s>>>(g, cn, n, G, ldg);
    return cudaGetLastError();
}

cudaError_t launch_sparse_to_dense(const int32_t *rows, const int8_t *signs, int64_t n, int nnz, double *G,
                                   int64_t ldg, cudaStream_t s) {
    note_launch();
    k_zero<<<grid_for(n * n, 256), 256, 0, s>>>(G, n, ldg);
    note_launch();
    k_sparse_dense<<<grid_for(n, 128), 128, 0, s>>>(rows, signs, n, nnz, G, ldg);
    return cudaGetLastError();
}

}  // namespace genp
