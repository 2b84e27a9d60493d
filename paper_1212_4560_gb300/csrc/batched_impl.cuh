// batched_impl.cuh -- kernels of the batched solves (one persistent launch
// carries many small randomized-GENP systems), included by one translation
// unit per right-hand-side class (batched_r*.cu) so they compile in parallel.
//
// Each CTA (256 threads) pops the next system from an atomic work queue
// (systems sorted largest first) and carries it through the method alone:
//   C = A G             FP32 register-tiled CTA GEMM (64 x 64 or 128 x 128
//                       output tiles, 4 x 4 or 8 x 8 per thread, operands
//                       staged in shared memory, next k-step prefetched into
//                       registers); a copy of C is kept as the Krylov
//                       operator
//   C = L U             right-looking GENP in blocks of 32 columns: the
//                       diagonal block by one warp in shared memory, the
//                       block column (L21 = C21 U11^{-1}) and block row
//                       (U12 = L11^{-1} C12) by per-thread substitution
//                       against it, the Schur update C22 -= L21 U12 by the
//                       CTA GEMM
//   y = U^{-1} L^{-1} b blocks of 32 rows: the solved part enters through a
//                       coalesced GEMV (warps split rows and columns, lanes
//                       reduce by recursive halving), then one warp solves
//                       the 32 x 32 diagonal block with shuffles
//   x = G y
//   GMRES-IR            r = b - A x in FP64; an FP32 GMRES (CGS2 Arnoldi,
//                       Givens rotations, at most 16 steps) on
//                       U^{-1} L^{-1} C d = U^{-1} L^{-1} r / s, then
//                       x += s G d in FP64; until the backward error is
//                       <= tol, fails to halve on two steps in a row, or
//                       after max_iter steps (the first step often gains
//                       little: the preconditioned residual the inner solve
//                       reduces is not the true one).
// FP32 elimination of A G without pivoting loses u32 times the element growth
// (about 1e3 .. 1e4 for Gaussian systems of order 512), so classic refinement
// with these factors often diverges; the Krylov inner solve recovers a
// correction of about 1e-3 relative accuracy per outer step regardless
// (Carson & Higham, SIAM J. Sci. Comput. 2018).
// The adjoint kernel reuses the FP32 factors: Lambda = L^{-T} U^{-T} G^T gX,
// refined in FP64 against A^T, then dA = -Lambda X^T, dB = Lambda.  No CTA
// ever waits for another (the queue is a single atomic counter), so a launch
// cannot deadlock, and every reduction runs in a fixed order, so a run is
// reproducible bit for bit.
#pragma once

#include "genp_internal.cuh"

#include <math.h>

namespace genp {
namespace bimpl {
namespace {   // internal to each including translation unit

constexpr int BT = 256;       // threads per CTA
constexpr int NW = BT / 32;   // warps per CTA
constexpr int NB = 32;        // factorization and solve block
constexpr int GK = 16;        // CTA GEMM k-step
constexpr int GP = 132;       // pitch (floats) of the GEMM's shared tiles
constexpr int KM = kBatchedKrylov;   // Krylov steps per inner solve
constexpr double kInnerTol = 1e-3;

template <int NR>
struct Kry {
    double H[KM + 1][KM][NR];   // Hessenberg matrix, rotated in place into R
    double g[KM + 1][NR];       // rotated right-hand side beta e_1
    double cs[KM][NR], sn[KM][NR];
    double h[KM + 1][NR];       // dot products of the current pass / the solution y
    double beta[NR];
    double scale[NR];           // power-of-two scale of each residual column
    double scale_prev[NR];      // ... of the last accepted iterate
    double sinv[NR];            // 1 / scale (0 where the scale is 0)
    float red[NW][KM + 1][NR];  // per-warp partial dot products
    float rinv[NR];             // reciprocal norms of the vector being normalized
    int done[NR];
};

template <int NR>
struct Smem {
    union {
        struct {
            float As[GK][GP];
            float Bs[GK][GP];
        } t;
        float part[NW][32][NR];   // partial sums of the triangular solves
    } u;
    float D[NB][NB + 1];          // diagonal block of the factorization
    Kry<NR> k;
};

template <int NR>
constexpr size_t smem_fixed() {
    return (sizeof(Smem<NR>) + 15) / 16 * 16;
}

struct Ctl {
    int idx;
    unsigned int cmax, umax;      // max |C|, max |U| (float bits)
    float min_piv, max_piv;
    long long breakdown;
    unsigned long long anorm;     // ||A||_inf (double bits)
    unsigned long long rn[16], xn[16], bn[16];
    double eta, eta_prev, eta_prev2;
    int stop, restore, mode;
};

__device__ __forceinline__ void smax_u64(unsigned long long *p, double v) {
    atomicMax(p, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ double u64d(unsigned long long v) { return __longlong_as_double((long long)v); }

__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

// v[0..31] hold this lane's partial sums of 32 quantities; returns the
// warp-wide sum of quantity `lane` (recursive halving: 31 shuffles).
template <typename T>
__device__ __forceinline__ T reduce_scatter32(T (&v)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
        const bool up = (lane & h) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const T send = up ? v[i] : v[i + h];
            const T keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
        }
    }
    return v[0];
}

// ---------------------------------------------------------------------------
// CTA GEMM: acc(r, c) = sum_k A(i0 + r, k) B(k, j0 + c) over one TS x TS tile.
// Loaders return 0 outside their matrix.
// ---------------------------------------------------------------------------

// element (r, k) of a row-major FP64 or FP32 matrix with bounds
struct LoadA {
    const void *p;
    bool f64;
    int64_t ld;
    int rows, cols;
    __device__ __forceinline__ float at(int r, int k) const {
        if (r >= rows || k >= cols) return 0.f;
        const int64_t i = (int64_t)r * ld + k;
        return f64 ? (float)static_cast<const double *>(p)[i] : static_cast<const float *>(p)[i];
    }
};
struct LoadF {
    const float *p;
    int64_t ld;
    int rows, cols;
    __device__ __forceinline__ float at(int r, int k) const {
        return (r < rows && k < cols) ? p[(int64_t)r * ld + k] : 0.f;
    }
};
// circulant B(k, c) = g[(k - c) mod n]
struct LoadCirc {
    const float *g;
    int n;
    __device__ __forceinline__ float at(int k, int c) const {
        if (k >= n || c >= n) return 0.f;
        int d = k - c;
        d += d < 0 ? n : 0;
        return g[d];
    }
};

template <int TS, class LA, class LB>
__device__ __forceinline__ void tile_mma(int i0, int j0, int K, const LA &la, const LB &lb,
                                         float (&acc)[TS / 16][TS / 16], float (*As)[GP], float (*Bs)[GP]) {
    constexpr int R = TS / 16;
    constexpr int AE = TS * GK / BT;   // elements per thread and k-step: 8 (TS 128) or 4 (TS 64)
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int ar = tid % TS, ak = (tid / TS) * AE;
    const int bk = tid / (TS / AE), bc = (tid % (TS / AE)) * AE;
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = 0.f;
    float ra[AE], rb[AE];
#pragma unroll
    for (int e = 0; e < AE; ++e) {
        ra[e] = la.at(i0 + ar, ak + e);
        rb[e] = lb.at(bk, j0 + bc + e);
    }
    for (int k0 = 0; k0 < K; k0 += GK) {
        __syncthreads();
#pragma unroll
        for (int e = 0; e < AE; ++e) As[ak + e][ar] = ra[e];
#pragma unroll
        for (int e = 0; e < AE; ++e) Bs[bk][bc + e] = rb[e];
        __syncthreads();
        if (k0 + GK < K) {
#pragma unroll
            for (int e = 0; e < AE; ++e) {
                ra[e] = la.at(i0 + ar, k0 + GK + ak + e);
                rb[e] = lb.at(k0 + GK + bk, j0 + bc + e);
            }
        }
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float a[R], b[R];
#pragma unroll
            for (int h = 0; h < R / 4; ++h) {
                const float4 av = *reinterpret_cast<const float4 *>(&As[kk][h * 64 + ty * 4]);
                const float4 bv = *reinterpret_cast<const float4 *>(&Bs[kk][h * 64 + tx * 4]);
                a[4 * h] = av.x, a[4 * h + 1] = av.y, a[4 * h + 2] = av.z, a[4 * h + 3] = av.w;
                b[4 * h] = bv.x, b[4 * h + 1] = bv.y, b[4 * h + 2] = bv.z, b[4 * h + 3] = bv.w;
            }
#pragma unroll
            for (int i = 0; i < R; ++i)
#pragma unroll
                for (int j = 0; j < R; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
    }
}

// thread's tile coordinates of accumulator (i, j)
__device__ __forceinline__ int tile_row(int i) { return (i / 4) * 64 + (threadIdx.x >> 4) * 4 + (i % 4); }
__device__ __forceinline__ int tile_col(int j) { return (j / 4) * 64 + (threadIdx.x & 15) * 4 + (j % 4); }

// C = A G (A FP64 or FP32, G dense or circulant), written to C and to the
// Krylov copy Cc; returns this thread's max |C|.
template <int TS, class LB>
__device__ __noinline__ float gemm_ag(const LoadA &la, const LB &lb, int n, float *C, float *Cc, float (*As)[GP], float (*Bs)[GP]) {
    float cm = 0.f;
    for (int i0 = 0; i0 < n; i0 += TS)
        for (int j0 = 0; j0 < n; j0 += TS) {
            float acc[TS / 16][TS / 16];
            tile_mma<TS>(i0, j0, n, la, lb, acc, As, Bs);
#pragma unroll
            for (int i = 0; i < TS / 16; ++i) {
                const int r = i0 + tile_row(i);
                if (r >= n) continue;
#pragma unroll
                for (int j = 0; j < TS / 16; ++j) {
                    const int c = j0 + tile_col(j);
                    if (c >= n) continue;
                    const int64_t e = (int64_t)r * n + c;
                    C[e] = acc[i][j];
                    Cc[e] = acc[i][j];
                    cm = fmaxf(cm, fabsf(acc[i][j]));
                }
            }
        }
    return cm;
}

// C -= A B for M x N x K row-major blocks (lda, ldb, ldc), one TS tile at a time.
template <int TS>
__device__ __noinline__ void gemm_sub(int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *C,
                                      int ldc, float (*As)[GP], float (*Bs)[GP]) {
    const LoadF la{A, lda, M, K};
    const LoadF lb{B, ldb, K, N};
    for (int i0 = 0; i0 < M; i0 += TS)
        for (int j0 = 0; j0 < N; j0 += TS) {
            float acc[TS / 16][TS / 16];
            tile_mma<TS>(i0, j0, K, la, lb, acc, As, Bs);
#pragma unroll
            for (int i = 0; i < TS / 16; ++i) {
                const int r = i0 + tile_row(i);
                if (r >= M) continue;
#pragma unroll
                for (int j = 0; j < TS / 16; ++j) {
                    const int c = j0 + tile_col(j);
                    if (c >= N) continue;
                    C[(int64_t)r * ldc + c] -= acc[i][j];
                }
            }
        }
}

template <int NR>
__device__ __forceinline__ void gemm_sub_any(int ts, int M, int N, int K, const float *A, int lda, const float *B,
                                             int ldb, float *C, int ldc, Smem<NR> &sm) {
    if (ts == 128 && M > 64 && N > 64)
        gemm_sub<128>(M, N, K, A, lda, B, ldb, C, ldc, sm.u.t.As, sm.u.t.Bs);
    else
        gemm_sub<64>(M, N, K, A, lda, B, ldb, C, ldc, sm.u.t.As, sm.u.t.Bs);
}

// ---------------------------------------------------------------------------
// Factorization (in place, FP32): blocked right-looking GENP, blocks of NB.
// ---------------------------------------------------------------------------
template <int NR>
__device__ __noinline__ void factor(float *C, int n, int ts, Smem<NR> &sm, Ctl &ctl) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float (*D)[NB + 1] = sm.D;
    float um = 0.f;
    for (int k0 = 0; k0 < n; k0 += NB) {
        const int kb = min(NB, n - k0);
        for (int e = tid; e < NB * NB; e += BT) {
            const int i = e / NB, j = e % NB;
            D[i][j] = (i < kb && j < kb) ? C[(int64_t)(k0 + i) * n + k0 + j] : 0.f;
        }
        __syncthreads();
        if (warp == 0) {
            // unblocked GENP of the diagonal block: lane i owns row i
            for (int j = 0; j < kb; ++j) {
                const float p = D[j][j];
                if (lane == 0) {
                    const float ap = fabsf(p);
                    if (!(ap > 0.f) || !isfinite(ap)) {
                        if (ctl.breakdown < 0) ctl.breakdown = k0 + j;
                    } else {
                        ctl.min_piv = fminf(ctl.min_piv, ap);
                        ctl.max_piv = fmaxf(ctl.max_piv, ap);
                    }
                }
                if (lane > j && lane < kb) {
                    const float l = D[lane][j] / p;
                    D[lane][j] = l;
                    for (int c = j + 1; c < kb; ++c) D[lane][c] = fmaf(-l, D[j][c], D[lane][c]);
                }
                __syncwarp();
            }
        }
        __syncthreads();
        for (int e = tid; e < kb * kb; e += BT) {
            const int i = e / kb, j = e % kb;
            C[(int64_t)(k0 + i) * n + k0 + j] = D[i][j];
            if (j >= i) um = fmaxf(um, fabsf(D[i][j]));
        }
        const int rem = n - k0 - kb;
        // block column L21 = C21 U11^{-1} (one row per item) and block row
        // U12 = L11^{-1} C12 (one column per item), against D
        for (int it = tid; it < 2 * rem; it += BT) {
            float x[NB];
            if (it < rem) {
                float *row = C + (int64_t)(k0 + kb + it) * n + k0;
#pragma unroll
                for (int j = 0; j < NB; ++j) x[j] = j < kb ? row[j] : 0.f;
#pragma unroll
                for (int j = 0; j < NB; ++j) {
                    if (j < kb) {
                        x[j] = x[j] / D[j][j];
#pragma unroll
                        for (int c = j + 1; c < NB; ++c) x[c] = fmaf(-x[j], D[j][c], x[c]);
                    }
                }
#pragma unroll
                for (int j = 0; j < NB; ++j)
                    if (j < kb) row[j] = x[j];
            } else {
                float *col = C + (int64_t)k0 * n + k0 + kb + (it - rem);
#pragma unroll
                for (int i = 0; i < NB; ++i) x[i] = i < kb ? col[(int64_t)i * n] : 0.f;
#pragma unroll
                for (int l = 0; l < NB; ++l)
#pragma unroll
                    for (int i = l + 1; i < NB; ++i) x[i] = fmaf(-D[i][l], x[l], x[i]);
#pragma unroll
                for (int i = 0; i < NB; ++i)
                    if (i < kb) {
                        col[(int64_t)i * n] = x[i];
                        um = fmaxf(um, fabsf(x[i]));
                    }
            }
        }
        __syncthreads();
        if (rem > 0) {   // C22 -= L21 U12
            const int o = k0 + kb;
            gemm_sub_any<NR>(ts, rem, rem, kb, C + (int64_t)o * n + k0, n, C + (int64_t)k0 * n + o, n,
                             C + (int64_t)o * n + o, n, sm);
        }
        __syncthreads();
    }
    for (int o = 16; o > 0; o >>= 1) um = fmaxf(um, __shfl_xor_sync(0xffffffffu, um, o));
    if (lane == 0) atomicMax(&ctl.umax, __float_as_uint(um));
    __syncthreads();
}

// Li = L^{-1} (unit lower) and Ui = U^{-1} (upper) of the factors in LU,
// stored in full (zeros off their triangle), by blocked substitution on the
// identity: row block k of Li is L_kk^{-1} times itself once the blocks above
// have been subtracted (right-looking, C -= A B by the CTA GEMM), and the
// same backwards for Ui.  2 n^3 / 3 flops; the inner solves then apply
// U^{-1} L^{-1} as two coalesced triangular GEMVs instead of 2 n / 32
// dependent block steps.
template <int NR>
__device__ __noinline__ void invert_factors(const float *LU, int n, int ts, float *Li, float *Ui, Smem<NR> &sm) {
    const int tid = threadIdx.x;
    float (*D)[NB + 1] = sm.D;
    for (int64_t e = tid; e < (int64_t)n * n; e += BT) {
        const float v = (e / n == e % n) ? 1.f : 0.f;
        Li[e] = v;
        Ui[e] = v;
    }
    for (int k0 = 0; k0 < n; k0 += NB) {
        const int kb = min(NB, n - k0), ke = k0 + kb;
        __syncthreads();
        for (int e = tid; e < NB * NB; e += BT) {
            const int i = e / NB, j = e % NB;
            D[i][j] = (i < kb && j < kb && j < i) ? LU[(int64_t)(k0 + i) * n + k0 + j] : 0.f;
        }
        __syncthreads();
        for (int c = tid; c < ke; c += BT) {   // rows k0..ke of Li, columns < ke
            float x[NB];
#pragma unroll
            for (int i = 0; i < NB; ++i) x[i] = i < kb ? Li[(int64_t)(k0 + i) * n + c] : 0.f;
#pragma unroll
            for (int l = 0; l < NB; ++l)
#pragma unroll
                for (int i = l + 1; i < NB; ++i) x[i] = fmaf(-D[i][l], x[l], x[i]);
#pragma unroll
            for (int i = 0; i < NB; ++i)
                if (i < kb) Li[(int64_t)(k0 + i) * n + c] = x[i];
        }
        __syncthreads();
        if (ke < n)
            gemm_sub_any<NR>(ts, n - ke, ke, kb, LU + (int64_t)ke * n + k0, n, Li + (int64_t)k0 * n, n,
                             Li + (int64_t)ke * n, n, sm);
    }
    for (int k0 = (n - 1) / NB * NB; k0 >= 0; k0 -= NB) {
        const int kb = min(NB, n - k0);
        __syncthreads();
        for (int e = tid; e < NB * NB; e += BT) {
            const int i = e / NB, j = e % NB;
            D[i][j] = (i < kb && j < kb && j >= i) ? LU[(int64_t)(k0 + i) * n + k0 + j] : 0.f;
        }
        __syncthreads();
        for (int c = k0 + tid; c < n; c += BT) {   // rows k0..k0+kb of Ui, columns >= k0
            float x[NB];
#pragma unroll
            for (int i = 0; i < NB; ++i) x[i] = i < kb ? Ui[(int64_t)(k0 + i) * n + c] : 0.f;
#pragma unroll
            for (int l = NB - 1; l >= 0; --l) {
                if (l < kb) {
                    x[l] = x[l] / D[l][l];
#pragma unroll
                    for (int i = 0; i < l; ++i) x[i] = fmaf(-D[i][l], x[l], x[i]);
                }
            }
#pragma unroll
            for (int i = 0; i < NB; ++i)
                if (i < kb) Ui[(int64_t)(k0 + i) * n + c] = x[i];
        }
        __syncthreads();
        if (k0 > 0)
            gemm_sub_any<NR>(ts, k0, n - k0, kb, LU + k0, n, Ui + (int64_t)k0 * n + k0, n, Ui + k0, n, sm);
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Triangular solves on an n x NR vector block y in shared memory.
// ---------------------------------------------------------------------------

// Row style (y = L^{-1} y or U^{-1} y): part[s][r][c] = sum over the
// segment s of the solved columns of LU[r0 + r][j] y[j][c].  Warps take
// (row chunk, column segment) units; each lane keeps 32 / NR rows x NR
// sums and the warp reduces them by recursive halving.
template <int NR>
constexpr int row_segments() {
    return NW / NR > 0 ? NW / NR : 1;
}

template <int NR>
__device__ void blk_gemv_rows(const float *LU, int n, int r0, int bs, int klo, int khi, const float *y,
                              float (*part)[32][NR]) {
    constexpr int RW = 32 / NR, RC = NR, S = row_segments<NR>();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int K = khi - klo;
    const int seg = ((K + S - 1) / S + 31) & ~31;
    for (int u = warp; u < RC * S; u += NW) {
        const int ch = u % RC, s = u / RC;
        const int jb = klo + s * seg, je = min(khi, jb + seg);
        float acc[32];
#pragma unroll
        for (int e = 0; e < 32; ++e) acc[e] = 0.f;
        for (int j = jb + lane; j < je; j += 32) {
            float yv[NR];
#pragma unroll
            for (int c = 0; c < NR; ++c) yv[c] = y[j * NR + c];
#pragma unroll
            for (int rr = 0; rr < RW; ++rr) {
                const int r = ch * RW + rr;
                const float a = r < bs ? LU[(int64_t)(r0 + r) * n + j] : 0.f;
#pragma unroll
                for (int c = 0; c < NR; ++c) acc[rr * NR + c] = fmaf(a, yv[c], acc[rr * NR + c]);
            }
        }
        const float v = reduce_scatter32(acc);
        part[s][ch * RW + lane / NR][lane % NR] = v;
    }
}

// Column style (y = U^{-T} y or L^{-T} y): lane r sums LU[j][r0 + r] y[j][c]
// over warp w's segment of the solved rows j (coalesced along the row).
template <int NR>
__device__ void blk_gemv_cols(const float *LU, int n, int r0, int bs, int klo, int khi, const float *y,
                              float (*part)[32][NR]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int K = khi - klo, seg = (K + NW - 1) / NW;
    const int jb = klo + warp * seg, je = min(khi, jb + seg);
    float acc[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[c] = 0.f;
    const bool ok = lane < bs;
#pragma unroll 4
    for (int j = jb; j < je; ++j) {
        const float a = ok ? LU[(int64_t)j * n + r0 + lane] : 0.f;
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] = fmaf(a, y[j * NR + c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < NR; ++c) part[warp][lane][c] = acc[c];
}

// One warp: y[r0 .. r0 + bs) = M^{-1} (y - sum_s part[s]) for the diagonal
// block M (lower or upper, unit or not) of LU or LU^T.
template <int NR>
__device__ void blk_diag(const float *LU, int n, int r0, int bs, float *y, const float (*part)[32][NR], int S,
                         bool lower, bool unit, bool trans) {
    const int lane = threadIdx.x & 31;
    float m[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        float v = 0.f;
        if (lane < bs && j < bs)
            v = trans ? LU[(int64_t)(r0 + j) * n + r0 + lane] : LU[(int64_t)(r0 + lane) * n + r0 + j];
        m[j] = v;
    }
    float t[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) {
        float s = lane < bs ? y[(r0 + lane) * NR + c] : 0.f;
        for (int q = 0; q < S; ++q) s -= part[q][lane][c];
        t[c] = s;
    }
    if (lower) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            if (j < bs) {
                if (!unit && lane == j)
#pragma unroll
                    for (int c = 0; c < NR; ++c) t[c] = t[c] / m[j];
#pragma unroll
                for (int c = 0; c < NR; ++c) {
                    const float yj = __shfl_sync(0xffffffffu, t[c], j);
                    if (lane > j) t[c] = fmaf(-m[j], yj, t[c]);
                }
            }
        }
    } else {
#pragma unroll
        for (int j = 31; j >= 0; --j) {
            if (j < bs) {
                if (!unit && lane == j)
#pragma unroll
                    for (int c = 0; c < NR; ++c) t[c] = t[c] / m[j];
#pragma unroll
                for (int c = 0; c < NR; ++c) {
                    const float yj = __shfl_sync(0xffffffffu, t[c], j);
                    if (lane < j) t[c] = fmaf(-m[j], yj, t[c]);
                }
            }
        }
    }
    if (lane < bs)
#pragma unroll
        for (int c = 0; c < NR; ++c) y[(r0 + lane) * NR + c] = t[c];
}

// y <- U^{-1} L^{-1} y (trans = false) or L^{-T} U^{-T} y (trans = true).
// Starts and ends with all of y visible to the CTA.
template <int NR>
__device__ __noinline__ void lu_solve(const float *LU, int n, float *y, Smem<NR> &sm, bool trans) {
    const int warp = threadIdx.x >> 5;
    const int nq = (n + NB - 1) / NB;
    for (int pass = 0; pass < 2; ++pass)
        for (int qq = 0; qq < nq; ++qq) {
            const int q = pass == 0 ? qq : nq - 1 - qq;
            const int r0 = q * NB, bs = min(NB, n - r0);
            const int klo = pass == 0 ? 0 : r0 + bs, khi = pass == 0 ? r0 : n;
            if (trans)
                blk_gemv_cols<NR>(LU, n, r0, bs, klo, khi, y, sm.u.part);
            else
                blk_gemv_rows<NR>(LU, n, r0, bs, klo, khi, y, sm.u.part);
            __syncthreads();
            if (warp == 0)
                blk_diag<NR>(LU, n, r0, bs, y, sm.u.part, trans ? NW : row_segments<NR>(), pass == 0,
                             trans ? pass == 1 : pass == 0, trans);
            __syncthreads();
        }
}

// ---------------------------------------------------------------------------
// Full matrix-vector products.
// ---------------------------------------------------------------------------

// Row style over all n rows: ep(r, c, sum_j M(r, j) x[j][c]) for x (n x NR)
// in shared memory; M(r, j) from the loader (FP32 arithmetic).
// tri = 0: all columns; 1: columns j < row0 + RW of each unit (lower
// triangular M, zeros above stored); 2: columns j >= row0 (upper).
template <int NR, class LM, class EP>
__device__ void gemv_rows(int n, const LM &m, const float *x, const EP &ep, int tri = 0) {
    constexpr int RW = 32 / NR;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int units = (n + RW - 1) / RW;
    for (int u = warp; u < units; u += NW) {
        const int row0 = u * RW;
        float acc[32];
#pragma unroll
        for (int e = 0; e < 32; ++e) acc[e] = 0.f;
        const int jlo = tri == 2 ? row0 : 0, jhi = tri == 1 ? min(n, row0 + RW) : n;
        for (int j = jlo + lane; j < jhi; j += 32) {
            float xv[NR];
#pragma unroll
            for (int c = 0; c < NR; ++c) xv[c] = x[j * NR + c];
#pragma unroll
            for (int rr = 0; rr < RW; ++rr) {
                const float a = m.at(row0 + rr, j);
#pragma unroll
                for (int c = 0; c < NR; ++c) acc[rr * NR + c] = fmaf(a, xv[c], acc[rr * NR + c]);
            }
        }
        const float v = reduce_scatter32(acc);
        const int r = row0 + lane / NR;
        if (r < n) ep(r, lane % NR, v);
    }
}

// Column style over all n outputs: ep(i, c, sum_j M(j, i) x(j, c)), lanes
// over i (coalesced along rows of M), one warp per 32 outputs, T arithmetic.
template <int NR, typename T, class LM, class LX, class EP>
__device__ void gemv_cols(int n, const LM &m, const LX &x, const EP &ep) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i0 = warp * 32; i0 < n; i0 += NW * 32) {
        const int i = i0 + lane;
        T acc[NR];
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] = T(0);
#pragma unroll 4
        for (int j = 0; j < n; ++j) {
            const T a = i < n ? m.at(j, i) : T(0);
#pragma unroll
            for (int c = 0; c < NR; ++c) acc[c] = fma_t(a, x(j, c), acc[c]);
        }
        if (i < n)
#pragma unroll
            for (int c = 0; c < NR; ++c) ep(i, c, acc[c]);
    }
}

// row loaders of the full products
struct RowsF {   // M(r, j) = p[r n + j], r < n
    const float *p;
    int n;
    __device__ __forceinline__ float at(int r, int j) const { return r < n ? p[(int64_t)r * n + j] : 0.f; }
};
struct RowsCirc {   // circulant M(r, j) = g[(r - j) mod n]
    const float *g;
    int n;
    __device__ __forceinline__ float at(int r, int j) const {
        if (r >= n) return 0.f;
        int d = r - j;
        d += d < 0 ? n : 0;
        return g[d];
    }
};
struct ColsF {   // M(j, i) = p[j n + i]
    const float *p;
    int n;
    __device__ __forceinline__ float at(int j, int i) const { return p[(int64_t)j * n + i]; }
};
struct ColsCirc {   // M(j, i) = G[j][i] = g[(j - i) mod n]
    const float *g;
    int n;
    __device__ __forceinline__ float at(int j, int i) const {
        int d = j - i;
        d += d < 0 ? n : 0;
        return g[d];
    }
};
struct ColsA64 {   // M(j, i) = A[j][i] in FP64
    const void *p;
    bool f64;
    int n;
    __device__ __forceinline__ double at(int j, int i) const {
        const int64_t e = (int64_t)j * n + i;
        return f64 ? static_cast<const double *>(p)[e] : (double)static_cast<const float *>(p)[e];
    }
};

// X (+)= s G y: y (n x NR) in shared memory, FP32 products added in FP64.
template <int NR>
__device__ __noinline__ void apply_g(const float *G, const float *g, int n, const float *y, double *X, int nr,
                        const double *scale, bool accumulate) {
    auto ep = [&](int r, int c, float v) {
        if (c >= nr) return;
        double *p = X + (int64_t)r * nr + c;
        const double d = scale ? (double)v * scale[c] : (double)v;
        *p = accumulate ? *p + d : d;
    };
    if (g)
        gemv_rows<NR>(n, RowsCirc{g, n}, y, ep);
    else
        gemv_rows<NR>(n, RowsF{G, n}, y, ep);
}

// R = B - A X in FP64 (R: n x NR scratch), column maxima of |R|, |X|, |B| into
// ctl; ||A||_inf too when `anorm`.
template <int NR>
__device__ __noinline__ void residual(const void *A, bool a64, int n, const double *B, const double *X, int nr, double *R,
                         bool anorm, Ctl &ctl) {
    constexpr int RW = 32 / NR;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int units = (n + RW - 1) / RW;
    for (int u = warp; u < units; u += NW) {
        const int row0 = u * RW;
        double acc[32];
#pragma unroll
        for (int e = 0; e < 32; ++e) acc[e] = 0.0;
        double rs[RW];
#pragma unroll
        for (int rr = 0; rr < RW; ++rr) rs[rr] = 0.0;
        for (int j = lane; j < n; j += 32) {
            double xv[NR];
#pragma unroll
            for (int c = 0; c < NR; ++c) xv[c] = c < nr ? X[(int64_t)j * nr + c] : 0.0;
#pragma unroll
            for (int rr = 0; rr < RW; ++rr) {
                const int r = row0 + rr;
                double a = 0.0;
                if (r < n) {
                    const int64_t e = (int64_t)r * n + j;
                    a = a64 ? static_cast<const double *>(A)[e] : (double)static_cast<const float *>(A)[e];
                }
                if (anorm) rs[rr] += fabs(a);
#pragma unroll
                for (int c = 0; c < NR; ++c) acc[rr * NR + c] = fma(a, xv[c], acc[rr * NR + c]);
            }
        }
        const double v = reduce_scatter32(acc);
        const int r = row0 + lane / NR, c = lane % NR;
        if (r < n) {
            double res = 0.0;
            if (c < nr) {
                const double b = B[(int64_t)r * nr + c];
                res = b - v;
                smax_u64(&ctl.rn[c], fabs(res));
                smax_u64(&ctl.xn[c], fabs(X[(int64_t)r * nr + c]));
                smax_u64(&ctl.bn[c], fabs(b));
            }
            R[r * NR + c] = res;
        }
        if (anorm) {
            double mx = 0.0;
#pragma unroll
            for (int rr = 0; rr < RW; ++rr) {
                double s = rs[rr];
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (row0 + rr < n) mx = fmax(mx, s);
            }
            if (lane == 0) smax_u64(&ctl.anorm, mx);
        }
    }
}

// Backward error max_c ||r_c|| / (||A|| ||x_c|| + ||b_c||) from ctl (thread 0).
__device__ double eta_of(const Ctl &ctl, int nr) {
    const double an = u64d(ctl.anorm);
    double e = 0.0;
    for (int c = 0; c < nr; ++c) {
        const double rn = u64d(ctl.rn[c]);
        double v = rn == 0.0 ? 0.0 : rn / (an * u64d(ctl.xn[c]) + u64d(ctl.bn[c]));
        if (!(v == v)) v = INFINITY;
        e = fmax(e, v);
    }
    return e;
}

// k.h[j][c] = sum_i V_j[i][c] b[i][c] for j < nj (V_j = V + j len, len = n NR).
template <int NR>
__device__ void multi_dots(const float *V, int nj, const float *b, int len, Kry<NR> &k) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float p[KM + 1];
#pragma unroll
    for (int j = 0; j <= KM; ++j) p[j] = 0.f;
    for (int e = tid; e < len; e += BT) {
        const float bv = b[e];
#pragma unroll
        for (int j = 0; j <= KM; ++j)
            if (j < nj) p[j] = fmaf(V[(int64_t)j * len + e], bv, p[j]);
    }
#pragma unroll
    for (int j = 0; j <= KM; ++j) {
        if (j < nj) {
            float s = p[j];
#pragma unroll
            for (int o = 16; o >= NR; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane < NR) k.red[warp][j][lane] = s;
        }
    }
    __syncthreads();
    for (int t = tid; t < nj * NR; t += BT) {
        const int j = t / NR, c = t % NR;
        double s = 0.0;
        for (int w = 0; w < NW; ++w) s += (double)k.red[w][j][c];
        k.h[j][c] = s;
    }
    __syncthreads();
}

// One inner GMRES solve: va <- d with M Cc d ~ M R / s (column scales s in
// k.scale), M = Ui Li the explicit inverse of the factors, or (exact) M
// applied by substitution with L and U.
// V: (KM + 1) x n x NR scratch.  Returns the Krylov steps taken.
// vb <- Ui (Li vb) (va is overwritten); all of vb visible on entry and exit.
template <int NR>
__device__ __forceinline__ void apply_inverse(const float *Li, const float *Ui, int n, float *va, float *vb) {
    gemv_rows<NR>(n, RowsF{Li, n}, vb, [&](int r, int c, float v) { va[r * NR + c] = v; }, 1);
    __syncthreads();
    gemv_rows<NR>(n, RowsF{Ui, n}, va, [&](int r, int c, float v) { vb[r * NR + c] = v; }, 2);
    __syncthreads();
}

template <int NR>
__device__ __noinline__ int inner_gmres(bool exact, const float *LU, const float *Li, const float *Ui, const float *Cc,
                                        int n, float *va, float *vb, float *V, const double *R, Smem<NR> &sm) {
    Kry<NR> &k = sm.k;
    const int tid = threadIdx.x, len = n * NR;
    auto precondition = [&]() {
        if (exact)
            lu_solve<NR>(LU, n, vb, sm, false);
        else
            apply_inverse<NR>(Li, Ui, n, va, vb);
    };
    if (tid < NR) k.sinv[tid] = k.scale[tid] > 0.0 ? 1.0 / k.scale[tid] : 0.0;   // powers of two: exact
    __syncthreads();
    for (int e = tid; e < len; e += BT) vb[e] = (float)(R[e] * k.sinv[e % NR]);
    __syncthreads();
    precondition();
    multi_dots<NR>(vb, 1, vb, len, k);
    if (tid < NR) {
        double b = sqrt(k.h[0][tid]);
        if (!(b < INFINITY)) b = 0.0;
        k.beta[tid] = b;
        k.g[0][tid] = b;
        k.done[tid] = !(b > 0.0);
        k.rinv[tid] = b > 0.0 ? (float)(1.0 / b) : 0.f;
    }
    __syncthreads();
    for (int e = tid; e < len; e += BT) {
        const float v = vb[e] * k.rinv[e % NR];
        va[e] = v;
        V[e] = v;
    }
    __syncthreads();
    int steps = 0;
    for (int kk = 0; kk < KM; ++kk) {
        gemv_rows<NR>(n, RowsF{Cc, n}, va, [&](int r, int c, float v) { vb[r * NR + c] = v; });
        __syncthreads();
        precondition();
        // classical Gram-Schmidt, twice
        for (int pass = 0; pass < 2; ++pass) {
            multi_dots<NR>(V, kk + 1, vb, len, k);
            if (tid < NR)
                for (int j = 0; j <= kk; ++j) k.H[j][kk][tid] = (pass ? k.H[j][kk][tid] : 0.0) + k.h[j][tid];
            for (int e = tid; e < len; e += BT) {
                const int c = e % NR;
                float w = vb[e];
                for (int j = 0; j <= kk; ++j) w = fmaf(-(float)k.h[j][c], V[(int64_t)j * len + e], w);
                vb[e] = w;
            }
            __syncthreads();
        }
        multi_dots<NR>(vb, 1, vb, len, k);
        if (tid < NR) {
            const int c = tid;
            double nrm = sqrt(k.h[0][c]);
            if (!(nrm < INFINITY)) nrm = 0.0;
            k.rinv[c] = nrm > 0.0 ? (float)(1.0 / nrm) : 0.f;
            k.H[kk + 1][kk][c] = nrm;
            for (int j = 0; j < kk; ++j) {
                const double a = k.H[j][kk][c], b = k.H[j + 1][kk][c];
                k.H[j][kk][c] = k.cs[j][c] * a + k.sn[j][c] * b;
                k.H[j + 1][kk][c] = -k.sn[j][c] * a + k.cs[j][c] * b;
            }
            const double a = k.H[kk][kk][c], b = k.H[kk + 1][kk][c];
            const double r = sqrt(a * a + b * b);
            const double cs = r > 0.0 ? a / r : 1.0, sn = r > 0.0 ? b / r : 0.0;
            k.cs[kk][c] = cs;
            k.sn[kk][c] = sn;
            k.H[kk][kk][c] = r;
            k.H[kk + 1][kk][c] = 0.0;
            k.g[kk + 1][c] = -sn * k.g[kk][c];
            k.g[kk][c] = cs * k.g[kk][c];
            k.done[c] = k.done[c] || !(fabs(k.g[kk + 1][c]) > kInnerTol * k.beta[c]) || !(nrm > 0.0);
        }
        __syncthreads();
        for (int e = tid; e < len; e += BT) {
            const float v = vb[e] * k.rinv[e % NR];
            va[e] = v;
            V[(int64_t)(kk + 1) * len + e] = v;
        }
        ++steps;
        bool all = true;
        for (int c = 0; c < NR; ++c) all = all && k.done[c];
        __syncthreads();
        if (all) break;
    }
    // y = R^{-1} g, then d = V y
    if (tid < NR) {
        const int c = tid;
        for (int i = steps - 1; i >= 0; --i) {
            double s = k.g[i][c];
            for (int l = i + 1; l < steps; ++l) s -= k.H[i][l][c] * k.h[l][c];
            k.h[i][c] = k.H[i][i][c] != 0.0 ? s / k.H[i][i][c] : 0.0;
        }
    }
    __syncthreads();
    for (int e = tid; e < len; e += BT) {
        const int c = e % NR;
        float d = 0.f;
        for (int j = 0; j < steps; ++j) d = fmaf((float)k.h[j][c], V[(int64_t)j * len + e], d);
        va[e] = d;
    }
    __syncthreads();
    return steps;
}

template <int NR>
__device__ __forceinline__ float *vec_a(unsigned char *raw) {
    return reinterpret_cast<float *>(raw + smem_fixed<NR>());
}

template <int NR>
__global__ void __launch_bounds__(BT, 2) k_batched(const BatchedArgs args) {
    const BatchDesc *d = args.desc;
    const int count = args.count, nmax = args.nmax, nr = args.nr, circ = args.circ, max_iter = args.max_iter;
    const int a64 = args.a64;
    const double tol = args.tol;
    int *counter = args.counter;
    const void *Apool = args.A;
    const double *Bpool = args.B;
    double *Xpool = args.X;
    float *Cpool = args.C;
    const float *Gpool = args.G, *gpool = args.g;
    float *scratch = args.scratch;
    const int64_t scratch_stride = args.stride;
    BatchStatus *stat = args.stat;
    extern __shared__ __align__(16) unsigned char smraw[];
    Smem<NR> &sm = *reinterpret_cast<Smem<NR> *>(smraw);
    const int64_t np = (nmax + 3) & ~3;
    float *va = vec_a<NR>(smraw), *vb = va + np * NR;
    __shared__ Ctl ctl;
    const int tid = threadIdx.x;
    // optional phase profile: thread 0 adds the SM cycles between barriers
    unsigned long long prof[kBatchedPhases] = {};
    long long tclk = clock64();
    auto lap = [&](int ph) {
        if (args.prof && tid == 0) {
            const long long t = clock64();
            prof[ph] += (unsigned long long)(t - tclk);
            tclk = t;
        }
    };
    // per-CTA scratch: Krylov copy of C, L^{-1}, U^{-1} (np^2 each), basis
    // (KM + 1) x np x NR, then FP64 np x NR each: the residual, the last
    // accepted x and its residual (np = nmax rounded up to 4: 16-byte offsets)
    float *Cc = scratch + (int64_t)blockIdx.x * scratch_stride;
    float *Li = Cc + np * np, *Ui = Li + np * np;
    float *V = Ui + np * np;
    double *R = reinterpret_cast<double *>(V + (int64_t)(KM + 1) * np * NR);
    double *Xprev = R + np * NR, *Rprev = Xprev + np * NR;
    while (true) {
        if (tid == 0) ctl.idx = atomicAdd(counter, 1);
        __syncthreads();
        const int idx = ctl.idx;
        if (idx >= count) break;
        const BatchDesc q = d[idx];
        const int n = (int)q.n, ts = q.nb;
        if (tid == 0) {
            ctl.breakdown = -1;
            ctl.min_piv = INFINITY;
            ctl.max_piv = 0.f;
            ctl.cmax = 0u;
            ctl.umax = 0u;
            ctl.anorm = 0ull;
        }
        __syncthreads();
        const void *A = a64 ? (const void *)((const double *)Apool + q.mat_off)
                            : (const void *)((const float *)Apool + q.mat_off);
        float *C = Cpool + q.mat_off;
        const float *G = circ ? nullptr : Gpool + q.mat_off;
        const float *g = circ ? gpool + q.g_off : nullptr;
        const double *B = Bpool + q.vec_off;
        double *X = Xpool + q.vec_off;

        // C = A G
        {
            const LoadA la{A, a64 != 0, n, n, n};
            float cm;
            if (g) {
                const LoadCirc lb{g, n};
                cm = ts == 128 ? gemm_ag<128>(la, lb, n, C, Cc, sm.u.t.As, sm.u.t.Bs)
                               : gemm_ag<64>(la, lb, n, C, Cc, sm.u.t.As, sm.u.t.Bs);
            } else {
                const LoadF lb{G, n, n, n};
                cm = ts == 128 ? gemm_ag<128>(la, lb, n, C, Cc, sm.u.t.As, sm.u.t.Bs)
                               : gemm_ag<64>(la, lb, n, C, Cc, sm.u.t.As, sm.u.t.Bs);
            }
            for (int o = 16; o > 0; o >>= 1) cm = fmaxf(cm, __shfl_xor_sync(0xffffffffu, cm, o));
            if ((tid & 31) == 0) atomicMax(&ctl.cmax, __float_as_uint(cm));
            __syncthreads();
        }
        lap(0);
        factor<NR>(C, n, ts, sm, ctl);
        lap(1);
        if (max_iter > 0) invert_factors<NR>(C, n, ts, Li, Ui, sm);
        lap(2);

        // x = G U^{-1} L^{-1} b
        const int len = n * NR;
        for (int e = tid; e < len; e += BT) {
            const int c = e % NR;
            vb[e] = c < nr ? (float)B[(int64_t)(e / NR) * nr + c] : 0.f;
        }
        __syncthreads();
        lu_solve<NR>(C, n, vb, sm, false);
        apply_g<NR>(G, g, n, vb, X, nr, nullptr, false);
        __syncthreads();
        lap(3);

        // GMRES-IR.  Mode 0: the explicit inverses precondition the inner
        // solves; after a stall or a step that raised eta (which is undone),
        // mode 1: substitution with L and U, slower but as accurate as the
        // factors; a stall or a bad step there ends the refinement.
        double eta0 = -1.0, eta = INFINITY;
        int it = 0, krylov = 0;
        if (tid == 0) {
            ctl.eta_prev = ctl.eta_prev2 = INFINITY;
            ctl.mode = 0;
        }
        for (;; ++it) {
            if (tid < 16) ctl.rn[tid] = ctl.xn[tid] = ctl.bn[tid] = 0ull;
            __syncthreads();
            residual<NR>(A, a64 != 0, n, B, X, nr, R, it == 0, ctl);
            __syncthreads();
            if (tid == 0) {
                double e = eta_of(ctl, nr);
                int restore = 0, stop = 0;
                if (it > 0 && !(e <= ctl.eta_prev)) {
                    restore = 1;
                    e = ctl.eta_prev;
                    if (ctl.mode == 0) {
                        ctl.mode = 1;
                        ctl.eta_prev2 = INFINITY;
                    } else {
                        stop = 1;
                    }
                } else {
                    const bool stalled = it > 1 && e > 0.5 * ctl.eta_prev && ctl.eta_prev > 0.5 * ctl.eta_prev2;
                    if (stalled && ctl.mode == 0) {
                        ctl.mode = 1;
                        ctl.eta_prev2 = INFINITY;
                    } else {
                        stop = stalled;
                        ctl.eta_prev2 = ctl.eta_prev;
                    }
                    ctl.eta_prev = e;
                }
                ctl.eta = e;
                ctl.restore = restore;
                ctl.stop = stop || (e <= tol) || it >= max_iter || ctl.breakdown >= 0;
            }
            if (tid < NR) {
                const double s = tid < nr ? u64d(ctl.rn[tid]) : 0.0;
                sm.k.scale[tid] = (s > 0.0 && s < INFINITY) ? ldexp(1.0, ilogb(s)) : 0.0;
            }
            __syncthreads();
            const int len = n * NR;
            if (ctl.restore) {   // back to the last accepted iterate and its residual
                for (int e = tid; e < len; e += BT) {
                    const int c = e % NR;
                    if (c < nr) X[(int64_t)(e / NR) * nr + c] = Xprev[e];
                    R[e] = Rprev[e];
                }
                if (tid < NR) sm.k.scale[tid] = sm.k.scale_prev[tid];
            } else if (!ctl.stop) {
                for (int e = tid; e < len; e += BT) {
                    const int c = e % NR;
                    Xprev[e] = c < nr ? X[(int64_t)(e / NR) * nr + c] : 0.0;
                    Rprev[e] = R[e];
                }
                if (tid < NR) sm.k.scale_prev[tid] = sm.k.scale[tid];
            }
            __syncthreads();
            lap(4);
            eta = ctl.eta;
            if (it == 0) eta0 = eta;
            if (ctl.stop) break;
            krylov += inner_gmres<NR>(ctl.mode != 0, C, Li, Ui, Cc, n, va, vb, V, R, sm);
            lap(5);
            apply_g<NR>(G, g, n, va, X, nr, sm.k.scale, true);
            __syncthreads();
            lap(6);
        }
        if (tid == 0) {
            BatchStatus st;
            st.breakdown_step = ctl.breakdown;
            st.min_abs_pivot = ctl.min_piv;
            st.max_abs_pivot = ctl.max_piv;
            st.max_abs_u = __uint_as_float(ctl.umax);
            st.max_abs_c = __uint_as_float(ctl.cmax);
            st.refine_iters = it;
            st.status = ctl.breakdown >= 0 ? GENP_ERR_BREAKDOWN : (eta <= tol ? GENP_OK : GENP_ERR_NOCONV);
            st.escalated = ctl.mode;
            st.krylov_steps = krylov;
            st.eta0 = eta0;
            st.eta = eta;
            stat[idx] = st;
        }
        __syncthreads();
        tclk = clock64();
    }
    if (args.prof && tid == 0)
        for (int p = 0; p < kBatchedPhases; ++p) args.prof[(int64_t)blockIdx.x * kBatchedPhases + p] = prof[p];
}

// Adjoint of every system: Lambda = A^{-T} gX = L^{-T} U^{-T} G^T gX with the
// FP32 factors, refined in FP64 (R = gX - A^T Lambda, Lambda += A^{-T} R)
// until the backward error is <= tol, fails to halve or after max_iter
// steps; dB = Lambda, dA = -Lambda X^T (FP32 output).
template <int NR>
__global__ void __launch_bounds__(BT, 2) k_batched_adjoint(const BatchedArgs args) {
    const BatchDesc *d = args.desc;
    const int count = args.count, nmax = args.nmax, nr = args.nr, circ = args.circ, max_iter = args.max_iter;
    const int a64 = args.a64;
    const double tol = args.tol;
    int *counter = args.counter;
    const void *Apool = args.A;
    const float *Cpool = args.C;
    const float *Gpool = args.G, *gpool = args.g;
    const double *gXpool = args.gX, *Xpool = args.X;
    double *Lpool = args.L, *dBpool = args.dB;
    float *dApool = args.dA;
    float *scratch = args.scratch;
    const int64_t scratch_stride = args.stride;
    extern __shared__ __align__(16) unsigned char smraw[];
    Smem<NR> &sm = *reinterpret_cast<Smem<NR> *>(smraw);
    const int64_t np = (nmax + 3) & ~3;
    float *va = vec_a<NR>(smraw), *vb = va + np * NR;
    __shared__ Ctl ctl;
    const int tid = threadIdx.x;
    double *R = reinterpret_cast<double *>(scratch + (int64_t)blockIdx.x * scratch_stride);   // nmax x NR
    while (true) {
        if (tid == 0) ctl.idx = atomicAdd(counter, 1);
        __syncthreads();
        const int idx = ctl.idx;
        if (idx >= count) break;
        const BatchDesc q = d[idx];
        const int n = (int)q.n, len = n * NR;
        const void *A = a64 ? (const void *)((const double *)Apool + q.mat_off)
                            : (const void *)((const float *)Apool + q.mat_off);
        const float *C = Cpool + q.mat_off;
        const float *G = circ ? nullptr : Gpool + q.mat_off;
        const float *g = circ ? gpool + q.g_off : nullptr;
        const double *gX = gXpool + q.vec_off;
        const double *X = Xpool + q.vec_off;
        double *Lam = Lpool + q.vec_off;
        // vb = G^T (v / s), v (n x nr, FP64, ld ldv; s powers of two): the
        // scaled input is rounded to FP32 into va once, then read from there
        auto gt_apply = [&](const double *v, int64_t ldv, const double *s) {
            if (tid < NR) sm.k.sinv[tid] = s ? (s[tid] > 0.0 ? 1.0 / s[tid] : 0.0) : 1.0;
            __syncthreads();
            for (int e = tid; e < len; e += BT) {
                const int c = e % NR;
                va[e] = c < nr ? (float)(v[(int64_t)(e / NR) * ldv + c] * sm.k.sinv[c]) : 0.f;
            }
            __syncthreads();
            auto x = [&](int j, int c) -> float { return va[j * NR + c]; };
            auto ep = [&](int i, int c, float val) { vb[i * NR + c] = val; };
            if (g)
                gemv_cols<NR, float>(n, ColsCirc{g, n}, x, ep);
            else
                gemv_cols<NR, float>(n, ColsF{G, n}, x, ep);
            __syncthreads();
        };
        gt_apply(gX, nr, nullptr);
        lu_solve<NR>(C, n, vb, sm, true);
        for (int e = tid; e < len; e += BT) {
            const int c = e % NR;
            if (c < nr) Lam[(int64_t)(e / NR) * nr + c] = (double)vb[e];
        }
        if (tid == 0) {
            ctl.eta_prev = INFINITY;
            ctl.anorm = 0ull;
        }
        __syncthreads();
        for (int it = 0;; ++it) {
            if (tid < 16) ctl.rn[tid] = ctl.xn[tid] = ctl.bn[tid] = 0ull;
            __syncthreads();
            // R = gX - A^T Lam (lanes over columns i of A), ||A^T||_inf once
            {
                const ColsA64 m{A, a64 != 0, n};
                const int lane = tid & 31, warp = tid >> 5;
                for (int i0 = warp * 32; i0 < n; i0 += NW * 32) {
                    const int i = i0 + lane;
                    double acc[NR];
#pragma unroll
                    for (int c = 0; c < NR; ++c) acc[c] = 0.0;
                    double cs = 0.0;
                    if (i < n) {
#pragma unroll 4
                        for (int j = 0; j < n; ++j) {
                            const double a = m.at(j, i);
                            cs += fabs(a);
#pragma unroll
                            for (int c = 0; c < NR; ++c)
                                acc[c] = fma(a, c < nr ? Lam[(int64_t)j * nr + c] : 0.0, acc[c]);
                        }
                        if (it == 0) smax_u64(&ctl.anorm, cs);
#pragma unroll
                        for (int c = 0; c < NR; ++c) {
                            double r = 0.0;
                            if (c < nr) {
                                r = gX[(int64_t)i * nr + c] - acc[c];
                                smax_u64(&ctl.rn[c], fabs(r));
                                smax_u64(&ctl.xn[c], fabs(Lam[(int64_t)i * nr + c]));
                                smax_u64(&ctl.bn[c], fabs(gX[(int64_t)i * nr + c]));
                            }
                            R[i * NR + c] = r;
                        }
                    }
                }
            }
            __syncthreads();
            if (tid == 0) {
                const double e = eta_of(ctl, nr);
                ctl.stop = (e <= tol) || (it > 0 && e > 0.5 * ctl.eta_prev) || it >= max_iter;
                ctl.eta_prev = e;
            }
            if (tid < NR) {
                const double s = tid < nr ? u64d(ctl.rn[tid]) : 0.0;
                sm.k.scale[tid] = (s > 0.0 && s < INFINITY) ? ldexp(1.0, ilogb(s)) : 0.0;
            }
            __syncthreads();
            if (ctl.stop) break;
            gt_apply(R, NR, sm.k.scale);
            lu_solve<NR>(C, n, vb, sm, true);
            for (int e = tid; e < len; e += BT) {
                const int c = e % NR;
                if (c < nr && sm.k.scale[c] > 0.0) Lam[(int64_t)(e / NR) * nr + c] += (double)vb[e] * sm.k.scale[c];
            }
            __syncthreads();
        }
        if (dBpool)
            for (int e = tid; e < n * nr; e += BT) dBpool[q.vec_off + e] = Lam[e];
        if (dApool) {
            // dA = -Lambda X^T with Lambda and X rounded to FP32 (in va, vb)
            for (int e = tid; e < len; e += BT) {
                const int c = e % NR, i = e / NR;
                va[e] = c < nr ? (float)Lam[(int64_t)i * nr + c] : 0.f;
                vb[e] = c < nr ? (float)X[(int64_t)i * nr + c] : 0.f;
            }
            __syncthreads();
            float *dA = dApool + q.mat_off;
            for (int64_t e = tid; e < (int64_t)n * n; e += BT) {
                const int i = (int)(e / n), j = (int)(e % n);
                float s = 0.f;
#pragma unroll
                for (int c = 0; c < NR; ++c) s = fmaf(va[i * NR + c], vb[j * NR + c], s);
                dA[e] = -s;
            }
        }
        __syncthreads();
    }
}

template <int NR>
size_t smem_bytes(int nmax) {
    return smem_fixed<NR>() + 2 * (size_t)((nmax + 3) & ~3) * NR * sizeof(float);
}

template <int NR>
int blocks_per_sm(int nmax) {
    const size_t sm = smem_bytes<NR>(nmax);
    cudaFuncSetAttribute(k_batched<NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(k_batched_adjoint<NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int b = 0, b2 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batched<NR>, BT, sm) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_batched_adjoint<NR>, BT, sm) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return b < b2 ? b : b2;
}

}  // namespace
}  // namespace bimpl
}  // namespace genp

// Entry points of one right-hand-side class NR (defined once per batched_r*.cu).
#define GENP_BATCHED_INSTANCE(NR)                                                                              \
    namespace genp {                                                                                           \
    int batched_blocks_per_sm_r##NR(int nmax) { return bimpl::blocks_per_sm<NR>(nmax); }                        \
    cudaError_t batched_launch_r##NR(const BatchedArgs &a, int grid, cudaStream_t s) {                          \
        bimpl::k_batched<NR><<<grid, bimpl::BT, bimpl::smem_bytes<NR>(a.nmax), s>>>(a);                         \
        return cudaGetLastError();                                                                             \
    }                                                                                                          \
    cudaError_t batched_adjoint_r##NR(const BatchedArgs &a, int grid, cudaStream_t s) {                         \
        bimpl::k_batched_adjoint<NR><<<grid, bimpl::BT, bimpl::smem_bytes<NR>(a.nmax), s>>>(a);                 \
        return cudaGetLastError();                                                                             \
    }                                                                                                          \
    }
