// lu.cu -- right-looking blocked GENP (Sec. 1.1; block Gaussian elimination,
// Thm. 2.2), in place on C:
//   for k0 = 0, nb, 2nb, ...
//     panel:  C11 = L11 U11           (one CTA, the nb x nb block in registers)
//     trsm:   U12 = L11^{-1} C12,  L21 = C21 U11^{-1}   (one launch, two roles)
//     schur:  C22 <- C22 - L21 U12    (tiled GEMM, the dominant cost, ~2n^3/3 flops)
// No row or column is ever exchanged.  A zero or non-finite pivot is
// recorded in the status word (first step wins) and elimination goes on.
#include "genp_internal.cuh"
#include "dfloat.cuh"

#include <math.h>

#include <type_traits>

namespace genp {
namespace {

constexpr int kTrsmW = 64;   // vectors (columns of C12 / rows of C21) per block-solve CTA

__global__ void k_status_reset(DevStatus *st) {
    st->breakdown_step = ~0ull;
    st->min_abs_pivot = 0x7FF0000000000000ull;  // +inf
    st->max_abs_pivot = 0ull;
    st->max_abs_u = 0ull;
    st->max_abs_c = 0ull;
}

template <typename T>
__global__ void k_maxabs(const T *C, int64_t n, int64_t ldc, unsigned long long *out) {
    double m = 0.0;
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x)
        for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
            const double v = fabs((double)C[r * ldc + c]);
            m = (v > m || isnan(v)) ? v : m;
        }
    for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_xor_sync(0xffffffffu, m, o);
        m = (w > m || isnan(w)) ? w : m;
    }
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(out, m);
}

// ---------------------------------------------------------------------------
// Register-blocked panel and block row / column solves: FP64 (TC = double),
// double-float (TC = dfloat: the sliced path, whose accuracy is set by its
// 47-bit products, on the FP32 pipe, which on GB300 is 64 times faster than
// the FP64 units) or FP32 (TC = float, the block solves of the FP32-storage
// paths).  Each thread keeps its share of the block in registers; the inner
// loops have no integer division.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double fms(double x, double l, double u) { return fma(-l, u, x); }
__device__ __forceinline__ float fms(float x, float l, float u) { return fmaf(-l, u, x); }
// x - l u in double-float: TwoProduct of the leading parts by FMA, TwoSum of
// x.hi and the product, the small terms gathered, one renormalization.
__device__ __forceinline__ dfloat fms(dfloat x, dfloat l, dfloat u) {
    const float p = l.hi * u.hi;
    const float pe = fmaf(l.hi, u.hi, -p) + fmaf(l.hi, u.lo, l.lo * u.hi);
    const float s = x.hi - p, bb = s - x.hi;
    const float err = (x.hi - (s - bb)) - (p + bb);
    return df_norm(s, (err + x.lo) - pe);
}
// The same on two entries at once with packed FP32 operations (hi and lo
// parts of the pair in float2 registers), the operations and roundings of
// the scalar form in the same order: np is -l.hi u.hi, formed from the
// negated leading part of the operand the pair shares, and a - b is an FMA
// of b by -1 and a.
__device__ __forceinline__ void fms2(float2 &xh, float2 &xl, float2 lh, float2 ll, float2 uh, float2 ul,
                                     float2 np) {
    const float2 m1 = make_float2(-1.0f, -1.0f);
    const float2 e1 = __ffma2_rn(lh, uh, np);                         // l.hi u.hi - p
    const float2 pe = __fadd2_rn(e1, __ffma2_rn(lh, ul, __fmul2_rn(ll, uh)));
    const float2 sm = __fadd2_rn(xh, np);                             // x.hi - p
    const float2 bb = __ffma2_rn(xh, m1, sm);                         // s - x.hi
    const float2 q2 = __ffma2_rn(__ffma2_rn(bb, m1, sm), m1, xh);     // x.hi - (s - bb)
    const float2 q3 = __ffma2_rn(np, m1, bb);                         // p + bb
    const float2 er = __fadd2_rn(__ffma2_rn(q3, m1, q2), xl);         // err + x.lo
    const float2 e = __ffma2_rn(pe, m1, er);                          // - pe
    const float2 hn = __fadd2_rn(sm, e);
    xh = hn;
    xl = __ffma2_rn(__ffma2_rn(sm, m1, hn), m1, e);                   // e - (hn - s)
}
__device__ __forceinline__ double shfl_idx(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ float shfl_idx(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ dfloat shfl_idx(dfloat v, int src) {
    v.hi = __shfl_sync(0xffffffffu, v.hi, src);
    v.lo = __shfl_sync(0xffffffffu, v.lo, src);
    return v;
}
// loads and stores between the storage type (double, or the double-float
// trailing matrix of the sliced path) and the compute type
template <typename TC> __device__ __forceinline__ TC ld_as(double v) { return TC(v); }
template <typename TC> __device__ __forceinline__ TC ld_as(dfloat v);
template <> __device__ __forceinline__ dfloat ld_as<dfloat>(dfloat v) { return v; }
template <typename TS> __device__ __forceinline__ TS st_as(double v) { return TS(v); }
template <typename TS> __device__ __forceinline__ TS st_as(dfloat v);
template <> __device__ __forceinline__ dfloat st_as<dfloat>(dfloat v) { return v; }
template <> __device__ __forceinline__ float st_as<float>(dfloat v) { return v.hi + v.lo; }
// magnitude for the growth statistics, without FP64 work for double-float
__device__ __forceinline__ double mag(double v) { return fabs(v); }
__device__ __forceinline__ float mag(float v) { return fabsf(v); }
__device__ __forceinline__ float mag(dfloat v) { return fabsf(v.hi); }

__device__ __forceinline__ void pivot_stats(DevStatus *st, int64_t step, double p) {
    const double ap = fabs(p);
    if (!(ap > 0.0) || !isfinite(ap)) {
        atomicMin(&st->breakdown_step, (unsigned long long)step);
    } else {
        atomic_min_nonneg(&st->min_abs_pivot, ap);
        atomic_max_nonneg(&st->max_abs_pivot, ap);
    }
}

// GENP of the kb x kb (kb <= 128) diagonal block at (k0, k0), by 32-column
// strips in shared memory (the block rounded up to whole strips, padded with
// the identity).  Per strip: (1) its 32 pivot steps with one block barrier
// each: the 8 threads of the pivot row publish the row's strip entries (its
// pivot's owner also the reciprocal in double-float), then every row below
// takes its multiplier from the thread that holds it (a shuffle inside the
// row's 8 threads, which keep 4 strip entries each in registers) and updates
// its strip entries; (2) the block row right of the strip, U12 = L11^{-1}
// A12, 8 threads per column with the substitution carried by shuffles; (3)
// the trailing block -= L21 U12 (K = 32), a register-tiled product over all
// threads.  The pivot steps touch only the strip; most of the arithmetic is
// in (3), without per-step barriers.  FP64 and double-float multiply by the
// pivot's reciprocal (an FP64 division per row costs a warp-wide sequence of
// FP64 operations each), FP32 divides.
constexpr int kPanelThreads = 1024, kPanelLd = 129;

// 1 / p in double-float by two Newton steps from the hardware's
// approximate single-precision reciprocal (r <- r + r (1 - p r), each step
// doubling the correct bits: ~22 -> 44 -> beyond the pair's 48), without
// the IEEE division's slow path.  FP32 keeps the pivot and divides by it
// (prcp below), as the unblocked recurrence does.
__device__ __forceinline__ dfloat panel_rcp(dfloat p) {
    float r0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(p.hi));
    dfloat r(r0);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const dfloat e = dfloat(1.0f) - p * r;
        r = r + r * e;
    }
    return r;
}
__device__ __forceinline__ float panel_rcp(float p) { return p; }
__device__ __forceinline__ dfloat panel_mult(dfloat x, dfloat rcp) { return x * rcp; }
__device__ __forceinline__ float panel_mult(float x, float p) { return x / p; }

// acc -= L21 U12 over the strip's 32 columns for the R x R outputs (rows
// e0 + ti + 32 a, columns e0 + tj + 32 b) of thread (ti, tj)
template <int R, typename TC>
__device__ __forceinline__ void panel_trailing(TC (*M)[kPanelLd], int s0, int e0, int ti, int tj) {
    TC acc[R][R];
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
        for (int b = 0; b < R; ++b) acc[a][b] = M[e0 + ti + 32 * a][e0 + tj + 32 * b];
#pragma unroll 4
    for (int k = 0; k < 32; ++k) {
        TC lv[R], uv[R];
#pragma unroll
        for (int a = 0; a < R; ++a) lv[a] = M[e0 + ti + 32 * a][s0 + k];
#pragma unroll
        for (int b = 0; b < R; ++b) uv[b] = M[s0 + k][e0 + tj + 32 * b];
#pragma unroll
        for (int a = 0; a < R; ++a)
#pragma unroll
            for (int b = 0; b < R; ++b) acc[a][b] = fms(acc[a][b], lv[a], uv[b]);
    }
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
        for (int b = 0; b < R; ++b) M[e0 + ti + 32 * a][e0 + tj + 32 * b] = acc[a][b];
}

// dynamic shared memory: the block's kbp rows (kb rounded up to 32), and
// for the FP32-pipe types the strip's multipliers (kbp x 33)
template <typename TC>
size_t panel_smem(int kb) {
    const size_t kbp = (size_t)((kb + 31) & ~31);
    return kbp * kPanelLd * sizeof(TC) + (std::is_same<TC, double>::value ? 0 : kbp * 33 * sizeof(TC));
}

template <typename TS, typename TC>
__global__ void __launch_bounds__(kPanelThreads, 1) k_panel_reg(TS *C, int64_t ldc, int64_t k0, int kb,
                                                                DevStatus *st) {
    extern __shared__ __align__(16) unsigned char smraw[];
    TC(*M)[kPanelLd] = reinterpret_cast<TC(*)[kPanelLd]>(smraw);
    __shared__ TC prow[2][32], prcp[2], piv[128];
    const int tid = threadIdx.x, lane = tid & 31;
    const int kbp = (kb + 31) & ~31;
    for (int idx = tid; idx < kbp * kbp; idx += kPanelThreads) {
        const int r = idx / kbp, c = idx % kbp;
        M[r][c] = (r < kb && c < kb) ? ld_as<TC>(C[(k0 + r) * ldc + k0 + c]) : TC(r == c ? 1.0 : 0.0);
    }
    __syncthreads();
    const int rho = tid >> 3, cq = tid & 7;       // strip role: row rho, strip columns cq + 8 j
    for (int s0 = 0; s0 < kbp; s0 += 32) {
        // ---- (1) the strip's pivot steps ----
        if constexpr (std::is_same<TC, double>::value) {
            const bool srow = rho >= s0 && rho < kbp;  // uniform per warp (4 rows per warp)
            TC sv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) sv[j] = srow ? M[rho][s0 + cq + 8 * j] : TC(0.0);
#pragma unroll 1
            for (int k = 0; k < 32; ++k) {
                const int pk = s0 + k, buf = k & 1;
                if (rho == pk) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) prow[buf][cq + 8 * j] = sv[j];
                    if (cq == (k & 7)) {
                        TC p = TC(0.0);
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if (j == (k >> 3)) p = sv[j];
                        prcp[buf] = TC(1.0) / p;   // one reciprocal per pivot, not a division per row
                        if (pk < kb) pivot_stats(st, k0 + pk, (double)p);
                    }
                }
                __syncthreads();
                TC l = TC(0.0);
                if (srow && rho > pk && cq == (k & 7)) {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (j == (k >> 3)) {
                            sv[j] = sv[j] * prcp[buf];
                            l = sv[j];
                        }
                }
                l = shfl_idx(l, (lane & ~7) | (k & 7));
                if (srow && rho > pk) {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (cq + 8 * j > k) sv[j] = fms(sv[j], l, prow[buf][cq + 8 * j]);
                }
            }
            if (srow)
#pragma unroll
                for (int j = 0; j < 4; ++j) M[rho][s0 + cq + 8 * j] = sv[j];
            __syncthreads();
        } else {
            // the strip in shared memory; thread (row rt, column group cg) of
            // 8 groups of 4 columns: a warp holds 32 rows of one group, so
            // whether a group still has columns to update is uniform per
            // warp.  Each thread forms its row's multiplier itself (FP32:
            // divides by the pivot; double-float: multiplies by its
            // reciprocal, which the thread that finishes the next pivot
            // forms); one barrier per step.  The multipliers go to Lm and into the strip
            // at its end (the other groups read column pk during the step).
            TC(*Lm)[33] = reinterpret_cast<TC(*)[33]>(&M[kbp][0]);
            const int rt = tid & 127, cg = tid >> 7;
            const bool srow = rt >= s0 && rt < kbp;      // uniform per warp
            if (tid == 0) {
                const TC p = M[s0][s0];
                piv[s0] = p;
                prcp[0] = panel_rcp(p);
            }
            __syncthreads();
#pragma unroll 1
            for (int k = 0; k < 32; ++k) {
                const int pk = s0 + k, buf = k & 1;
                if (srow && rt > pk) {
                    const TC l = panel_mult(M[rt][pk], prcp[buf]);
                    if (cg == 0) Lm[rt][k] = l;
                    if (4 * cg + 3 > k) {                // uniform per warp
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int c = s0 + 4 * cg + j;
                            if (c > pk) {
                                const TC v = fms(M[rt][c], l, M[pk][c]);
                                M[rt][c] = v;
                                if (rt == pk + 1 && c == pk + 1 && k < 31) {   // the next pivot
                                    piv[pk + 1] = v;
                                    prcp[buf ^ 1] = panel_rcp(v);
                                }
                            }
                        }
                    }
                }
                __syncthreads();
            }
            // the multipliers into the strip (below each pivot)
            for (int idx = tid; idx < 32 * 128; idx += kPanelThreads) {
                const int r = idx >> 5, k = idx & 31;
                if (r > s0 + k && r < kbp) M[r][s0 + k] = Lm[r][k];
            }
            __syncthreads();
        }
        const int e0 = s0 + 32, W = kbp - e0;
        if (W <= 0) break;
        // ---- (2) the block row: L11 x = a for each column e0 + col ----
        {
            const int col = tid >> 3, g = tid & 7;      // rows s0 + g + 8 m
            if (col < W) {                               // uniform per warp (4 columns per warp)
                TC x[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) x[m] = M[s0 + g + 8 * m][e0 + col];
#pragma unroll
                for (int b = 0; b < 4; ++b) {
#pragma unroll 1
                    for (int kk = 0; kk < 8; ++kk) {
                        const int k = 8 * b + kk;
                        const TC xk = shfl_idx(x[b], (lane & ~7) | kk);
                        if (g > kk) x[b] = fms(x[b], M[s0 + g + 8 * b][s0 + k], xk);
#pragma unroll
                        for (int m = b + 1; m < 4; ++m) x[m] = fms(x[m], M[s0 + g + 8 * m][s0 + k], xk);
                    }
                }
#pragma unroll
                for (int m = 0; m < 4; ++m) M[s0 + g + 8 * m][e0 + col] = x[m];
            }
        }
        __syncthreads();
        // ---- (3) the trailing block ----
        const int ti = tid >> 5, tj = tid & 31;
        if (W == 96) panel_trailing<3>(M, s0, e0, ti, tj);
        else if (W == 64) panel_trailing<2>(M, s0, e0, ti, tj);
        else panel_trailing<1>(M, s0, e0, ti, tj);
        __syncthreads();
    }
    if constexpr (!std::is_same<TC, double>::value) {
        // the pivots' statistics, off the pivot steps' path
        if (tid < 32)
            for (int k = tid; k < kb; k += 32) pivot_stats(st, k0 + k, (double)piv[k]);
    }
    using MT = decltype(mag(TC()));
    MT umax = 0;
    for (int idx = tid; idx < kb * kb; idx += kPanelThreads) {
        const int r = idx / kb, c = idx % kb;
        C[(k0 + r) * ldc + k0 + c] = st_as<TS>(M[r][c]);
        if (c >= r) {
            const MT av = mag(M[r][c]);
            umax = (av > umax || isnan(av)) ? av : umax;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const MT w = __shfl_xor_sync(0xffffffffu, umax, o);
        umax = (w > umax || isnan(w)) ? w : umax;
    }
    if (lane == 0) atomic_max_nonneg(&st->max_abs_u, (double)umax);
}

// blockIdx.y == 0: U12 = L11^{-1} C12 on columns [c0, c0 + 64)
// blockIdx.y == 1: L21 = C21 U11^{-1} on rows    [c0, c0 + 64)
// 64 vectors (columns of C12, rows of C21) per CTA of 1024 threads, 16
// threads per vector in one half-warp: thread g holds entries g + 16 m
// (m < 8, entry m in the m-th 16-block of the vector) in registers.  The
// substitution runs by 16-blocks: at step k = 16 b + kk the solved entry k
// reaches the vector's other threads by a shuffle, which update their entry
// of block b (below k) and every entry of the blocks after it; the blocks
// are unrolled, so a step costs the updates still to do and nothing for the
// blocks already solved (no per-entry conditions), and the step loop stays
// rolled (small code).  The kb x kb (kb <= 128) diagonal block sits in
// shared memory (row stride kbq + 1, kbq = kb rounded up to 16), padded
// with the identity, so a ragged last block needs no bounds checks.  32 warps per SM hide the latency of the
// dependent double-float operations.
constexpr int kTrsmThreads = 1024, kTpv = 16, kEpt = 128 / kTpv;
// dynamic shared memory of a block solve: the diagonal block rounded up to 16
// (double-float: hi and lo planes of the block as the packed solve reads
// it, [k][pair][thread][2], and the reciprocal pivots)
template <typename TC>
size_t trsm_smem(int kb) {
    const int kbq = (kb + kTpv - 1) / kTpv * kTpv;
    if (std::is_same<TC, dfloat>::value) {
        const int np = (kbq / kTpv + 1) / 2;
        return (size_t)kbq * np * kTpv * 2 * sizeof(float2) + (size_t)kbq * sizeof(dfloat);
    }
    return (size_t)kbq * (kbq + 1) * sizeof(TC);
}
// The vectors a block-solve launch takes: rows [l_beg, l_end) of the block
// column (L role) and columns [u_beg, u_end) of the block row (U role), 64
// per CTA, the L role's CTAs first.
struct TrsmRange {
    int64_t l_beg, l_end, u_beg, u_end;
};
__host__ __device__ __forceinline__ int trsm_l_ctas(const TrsmRange &rg) {
    return rg.l_end > rg.l_beg ? (int)((rg.l_end - rg.l_beg + kTrsmW - 1) / kTrsmW) : 0;
}
__host__ __device__ __forceinline__ int trsm_u_ctas(const TrsmRange &rg) {
    return rg.u_end > rg.u_beg ? (int)((rg.u_end - rg.u_beg + kTrsmW - 1) / kTrsmW) : 0;
}
// this CTA's role, first vector and vector count
__device__ __forceinline__ void trsm_cta(const TrsmRange &rg, bool &role_u, int64_t &c0, int &w) {
    const int nbl = trsm_l_ctas(rg);
    role_u = (int)blockIdx.x >= nbl;
    c0 = role_u ? rg.u_beg + (int64_t)((int)blockIdx.x - nbl) * kTrsmW : rg.l_beg + (int64_t)blockIdx.x * kTrsmW;
    w = (int)min((int64_t)kTrsmW, (role_u ? rg.u_end : rg.l_end) - c0);
}
template <typename TS>
__device__ __forceinline__ void trsm_df(TS *C, int64_t ldc, TrsmRange rg, int64_t k0, int kb, DevStatus *st,
                                        unsigned char *smraw);
template <typename TS, typename TC>
__global__ void __launch_bounds__(kTrsmThreads, 1) k_trsm_reg(TS *C, int64_t ldc, TrsmRange rg, int64_t k0, int kb,
                                                              DevStatus *st) {
    extern __shared__ __align__(16) unsigned char smraw[];
    if constexpr (std::is_same<TC, dfloat>::value) {
        trsm_df<TS>(C, ldc, rg, k0, kb, st, smraw);
        return;
    }
    TC *T = reinterpret_cast<TC *>(smraw);
    const int nq = (kb + kTpv - 1) / kTpv, kbq = kTpv * nq, ld = kbq + 1;   // the block rounded up to 16
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int v = tid / kTpv, g = tid % kTpv;
    bool role_u;
    int64_t c0;
    int w;
    trsm_cta(rg, role_u, c0, w);
    if (w <= 0) return;
    for (int r = warp; r < kbq; r += kTrsmThreads / 32)
        for (int c = lane; c < kbq; c += 32)
            T[r * ld + c] = (r < kb && c < kb) ? ld_as<TC>(C[(k0 + r) * ldc + k0 + c]) : TC(r == c ? 1.0 : 0.0);
    __syncthreads();
    // the L role divides by u_jj at every step: in FP64 and double-float by
    // reciprocals formed once (an FP64 division is a sequence of operations
    // that a whole warp issues for its one dividing lane, at 1/64 of the
    // FP32 rate on this GPU); FP32 divides
    constexpr bool kRcp = !std::is_same<TC, float>::value;
    if (kRcp && !role_u && tid < kbq) {
        const TC one(1.0);
        T[tid * ld + tid] = one / T[tid * ld + tid];
    }
    __syncthreads();
    const bool valid = v < w;
    const int base = lane & ~(kTpv - 1);
    TC x[kEpt];
    if (role_u) {
        // L11 x = c, L11 unit lower: x_r -= l_rk x_k for r > k
#pragma unroll
        for (int m = 0; m < kEpt; ++m) {
            const int r = g + kTpv * m;
            x[m] = (valid && r < kb) ? ld_as<TC>(C[(k0 + r) * ldc + c0 + v]) : TC(0.0);
        }
#pragma unroll
        for (int b = 0; b < kEpt; ++b) {
            if (b >= nq) break;
#pragma unroll 1
            for (int kk = 0; kk < kTpv; ++kk) {
                const int k = kTpv * b + kk;
                const TC xk = shfl_idx(x[b], base | kk);       // entry k, final
                if (g > kk) x[b] = fms(x[b], T[(g + kTpv * b) * ld + k], xk);
#pragma unroll
                for (int m = b + 1; m < kEpt; ++m)
                    if (m < nq) x[m] = fms(x[m], T[(g + kTpv * m) * ld + k], xk);   // (uniform) past kb: padding
            }
        }
        using MT = decltype(mag(TC()));
        MT xmax = 0;
#pragma unroll
        for (int m = 0; m < kEpt; ++m) {
            const int r = g + kTpv * m;
            if (valid && r < kb) {
                C[(k0 + r) * ldc + c0 + v] = st_as<TS>(x[m]);
                const MT av = mag(x[m]);
                xmax = (av > xmax || isnan(av)) ? av : xmax;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const MT q = __shfl_xor_sync(0xffffffffu, xmax, o);
            xmax = (q > xmax || isnan(q)) ? q : xmax;
        }
        if (lane == 0) atomic_max_nonneg(&st->max_abs_u, (double)xmax);
    } else {
        // x U11 = c, U11 upper: x_j = (c_j - sum_{i<j} x_i u_ij) / u_jj
#pragma unroll
        for (int m = 0; m < kEpt; ++m) {
            const int c = g + kTpv * m;
            x[m] = (valid && c < kb) ? ld_as<TC>(C[(c0 + v) * ldc + k0 + c]) : TC(0.0);
        }
#pragma unroll
        for (int b = 0; b < kEpt; ++b) {
            if (b >= nq) break;
#pragma unroll 1
            for (int kk = 0; kk < kTpv; ++kk) {
                const int j = kTpv * b + kk;
                if (g == kk) x[b] = kRcp ? x[b] * T[j * ld + j] : x[b] / T[j * ld + j];   // l_vj = x_vj / u_jj
                const TC xj = shfl_idx(x[b], base | kk);
                if (g > kk) x[b] = fms(x[b], xj, T[j * ld + g + kTpv * b]);
#pragma unroll
                for (int m = b + 1; m < kEpt; ++m)
                    if (m < nq) x[m] = fms(x[m], xj, T[j * ld + g + kTpv * m]);
            }
        }
#pragma unroll
        for (int m = 0; m < kEpt; ++m) {
            const int c = g + kTpv * m;
            if (valid && c < kb) C[(c0 + v) * ldc + k0 + c] = st_as<TS>(x[m]);
        }
    }
}

// The double-float block solve on packed FP32 pairs: the same substitution
// and roundings as the kernel above, each thread's eight entries held as four
// pairs (2p, 2p + 1) of hi and lo parts, every update of a pair one packed
// double-float multiply-subtract (half the FP32 instructions).  The block's
// operand of entry c = g + 16 m at step k (L11[c][k] for the block row,
// U11[k][c] for the block column) sits at [k][m / 2][g][m % 2] of a hi and a
// lo plane, so a thread reads a pair with one 8-byte load and a half-warp's
// loads are contiguous; past the block the planes hold the identity.
template <typename TS>
__device__ __forceinline__ void trsm_df(TS *C, int64_t ldc, TrsmRange rg, int64_t k0, int kb, DevStatus *st,
                                        unsigned char *smraw) {
    const int nq = (kb + kTpv - 1) / kTpv, kbq = kTpv * nq, np = (nq + 1) / 2, span = 2 * kTpv * np;
    float2 *Ph = reinterpret_cast<float2 *>(smraw);
    float2 *Pl = Ph + (size_t)kbq * np * kTpv;
    dfloat *rd = reinterpret_cast<dfloat *>(Pl + (size_t)kbq * np * kTpv);
    const int tid = threadIdx.x, lane = tid & 31;
    const int v = tid / kTpv, g = tid % kTpv;
    bool role_u;
    int64_t c0;
    int w;
    trsm_cta(rg, role_u, c0, w);
    if (w <= 0) return;
    for (int idx = tid; idx < kbq * span; idx += kTrsmThreads) {
        // the global reads run along a row of C: k fastest for the block row's
        // operand (a column of L11), c fastest for the block column's (a row of U11)
        const int k = role_u ? idx % kbq : idx / span, c = role_u ? idx / kbq : idx % span;
        const int r = role_u ? c : k, cc = role_u ? k : c;
        const dfloat t = (r < kb && cc < kb) ? ld_as<dfloat>(C[(k0 + r) * ldc + k0 + cc])
                                             : dfloat(r == cc ? 1.0f : 0.0f);
        const int m = c / kTpv, gg = c % kTpv;
        const size_t at = ((size_t)k * np + (m >> 1)) * kTpv + gg;
        reinterpret_cast<float *>(Ph + at)[m & 1] = t.hi;
        reinterpret_cast<float *>(Pl + at)[m & 1] = t.lo;
    }
    if (!role_u && tid < kbq) {
        const dfloat ujj = tid < kb ? ld_as<dfloat>(C[(k0 + tid) * ldc + k0 + tid]) : dfloat(1.0f);
        rd[tid] = dfloat(1.0) / ujj;
    }
    __syncthreads();
    const bool valid = v < w;
    const int base = lane & ~(kTpv - 1);
    float2 xh[kEpt / 2], xl[kEpt / 2];
#pragma unroll
    for (int p = 0; p < kEpt / 2; ++p) {
        dfloat a[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = g + kTpv * (2 * p + h);
            a[h] = (valid && e < kb) ? ld_as<dfloat>(role_u ? C[(k0 + e) * ldc + c0 + v] : C[(c0 + v) * ldc + k0 + e])
                                     : dfloat(0.0f);
        }
        xh[p] = make_float2(a[0].hi, a[1].hi);
        xl[p] = make_float2(a[0].lo, a[1].lo);
    }
#pragma unroll
    for (int b = 0; b < kEpt; ++b) {
        if (b >= nq) break;
        const int pb = b >> 1;
#pragma unroll 1
        for (int kk = 0; kk < kTpv; ++kk) {
            const int k = kTpv * b + kk;
            if (!role_u && g == kk) {
                // l_vk = x_vk / u_kk by the reciprocal pivot
                dfloat xb((b & 1) ? xh[pb].y : xh[pb].x);
                xb.lo = (b & 1) ? xl[pb].y : xl[pb].x;
                xb = xb * rd[k];
                if (b & 1) {
                    xh[pb].y = xb.hi;
                    xl[pb].y = xb.lo;
                } else {
                    xh[pb].x = xb.hi;
                    xl[pb].x = xb.lo;
                }
            }
            // entry k, final
            const float kh = __shfl_sync(0xffffffffu, (b & 1) ? xh[pb].y : xh[pb].x, base | kk);
            const float kl = __shfl_sync(0xffffffffu, (b & 1) ? xl[pb].y : xl[pb].x, base | kk);
            const float2 bh = make_float2(kh, kh), bl = make_float2(kl, kl);
            const float2 *ph = Ph + (size_t)k * np * kTpv + g, *pl = Pl + (size_t)k * np * kTpv + g;
            // block row: x -= L11[.][k] x_k (l varies, u = x_k); block column:
            // x -= x_k U11[k][.] (l = x_k, u varies)
            auto upd = [&](float2 &h, float2 &l, int p) {
                const float2 th = ph[p * kTpv], tl = pl[p * kTpv];
                if (role_u) fms2(h, l, th, tl, bh, bl, __fmul2_rn(th, make_float2(-kh, -kh)));
                else fms2(h, l, bh, bl, th, tl, __fmul2_rn(make_float2(-kh, -kh), th));
            };
            {
                // the pair of entry b: b itself below the step's row only
                float2 h = xh[pb], l = xl[pb];
                upd(h, l, pb);
                const bool below = g > kk;
                if (b & 1) {
                    xh[pb].y = below ? h.y : xh[pb].y;
                    xl[pb].y = below ? l.y : xl[pb].y;
                } else {
                    xh[pb].x = below ? h.x : xh[pb].x;
                    xl[pb].x = below ? l.x : xl[pb].x;
                    xh[pb].y = h.y;
                    xl[pb].y = l.y;
                }
            }
#pragma unroll
            for (int p = pb + 1; p < kEpt / 2; ++p)
                if (p < np) upd(xh[p], xl[p], p);   // (uniform) past kb: padding
        }
    }
    float xmax = 0.0f;
#pragma unroll
    for (int p = 0; p < kEpt / 2; ++p)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = g + kTpv * (2 * p + h);
            if (valid && e < kb) {
                dfloat a(h ? xh[p].y : xh[p].x);
                a.lo = h ? xl[p].y : xl[p].x;
                if (role_u) {
                    C[(k0 + e) * ldc + c0 + v] = st_as<TS>(a);
                    const float av = mag(a);
                    xmax = (av > xmax || isnan(av)) ? av : xmax;
                } else {
                    C[(c0 + v) * ldc + k0 + e] = st_as<TS>(a);
                }
            }
        }
    if (role_u) {
        for (int o = 16; o > 0; o >>= 1) {
            const float q = __shfl_xor_sync(0xffffffffu, xmax, o);
            xmax = (q > xmax || isnan(q)) ? q : xmax;
        }
        if (lane == 0) atomic_max_nonneg(&st->max_abs_u, (double)xmax);
    }
}

// one step of the blocked factorization's panel work: the diagonal block at
// (i0, i0) (panel_only), then the block row and column beside it (trsm_only)
template <typename TS, typename TC>
cudaError_t panel_attrs() {
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(k_trsm_reg<TS, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)trsm_smem<TC>(128));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_panel_reg<TS, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)panel_smem<TC>(128));
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    return cudaSuccess;
}
template <typename TS, typename TC>
cudaError_t panel_only(TS *C, int64_t ldc, int64_t i0, int kb, DevStatus *st, cudaStream_t s) {
    cudaError_t e = panel_attrs<TS, TC>();
    if (e != cudaSuccess) return e;
    auto *ev = profile_class_slot(kProfFactorAux, 2.0 / 3.0 * (double)kb * kb * kb);
    prof_begin(ev, s);
    note_launch();
    k_panel_reg<TS, TC><<<1, kPanelThreads, panel_smem<TC>(kb), s>>>(C, ldc, i0, kb, st);
    prof_end(ev, s);
    return cudaGetLastError();
}
template <typename TS, typename TC>
cudaError_t trsm_range(TS *C, int64_t ldc, TrsmRange rg, int64_t i0, int kb, DevStatus *st, cudaStream_t s) {
    const int ctas = trsm_l_ctas(rg) + trsm_u_ctas(rg);
    if (ctas <= 0) return cudaSuccess;
    cudaError_t e = panel_attrs<TS, TC>();
    if (e != cudaSuccess) return e;
    const double vecs = (double)((rg.l_end > rg.l_beg ? rg.l_end - rg.l_beg : 0) +
                                 (rg.u_end > rg.u_beg ? rg.u_end - rg.u_beg : 0));
    // kb^2 flops per vector of length kb
    auto *ev = profile_class_slot(kProfFactorAux, (double)kb * kb * vecs);
    prof_begin(ev, s);
    note_launch();
    k_trsm_reg<TS, TC><<<ctas, kTrsmThreads, trsm_smem<TC>(kb), s>>>(C, ldc, rg, i0, kb, st);
    prof_end(ev, s);
    return cudaGetLastError();
}
// the whole block row and block column beside the diagonal block at i0
template <typename TS, typename TC>
cudaError_t trsm_only(TS *C, int64_t ldc, int64_t n, int64_t i0, int kb, DevStatus *st, cudaStream_t s) {
    const int64_t j0 = i0 + kb;
    if (n - j0 <= 0) return cudaSuccess;
    return trsm_range<TS, TC>(C, ldc, TrsmRange{j0, n, j0, n}, i0, kb, st, s);
}
template <typename TS, typename TC>
cudaError_t panel_and_trsm(TS *C, int64_t ldc, int64_t n, int64_t i0, int kb, DevStatus *st, cudaStream_t s) {
    cudaError_t e = panel_only<TS, TC>(C, ldc, i0, kb, st, s);
    return e == cudaSuccess ? trsm_only<TS, TC>(C, ldc, n, i0, kb, st, s) : e;
}

template <typename TS, typename TC>
cudaError_t factor_typed(genp_factors *F, cudaStream_t s) {
    TS *C = static_cast<TS *>(F->C);
    const int64_t n = F->n, ldc = F->ldc;
    const int nb = (int)F->nb;
    note_launch();
    k_maxabs<TS><<<152 * 4, 256, 0, s>>>(C, n, ldc, &F->st->max_abs_c);
    for (int64_t k0 = 0; k0 < n; k0 += nb) {
        const int kb = (int)(n - k0 < nb ? n - k0 : nb);
        const int64_t rem = n - k0 - kb;
        cudaError_t e = panel_and_trsm<TS, TC>(C, ldc, n, k0, kb, F->st, s);
        if (e != cudaSuccess) return e;
        if (rem <= 0) break;
        TS *L21 = C + (k0 + kb) * ldc + k0;
        TS *U12 = C + k0 * ldc + k0 + kb;
        TS *A22 = C + (k0 + kb) * ldc + k0 + kb;
        e = gemm<TS>(rem, rem, kb, TS(-1), L21, ldc, false, U12, ldc, TS(1), A22, ldc, A22, ldc, nullptr, s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// Mixed precision (GENP_BF16, GENP_BF16X3, GENP_FP8_E4M3): C is the FP32
// master copy.  The diagonal block is factored in double-float (FP64-class
// pivots, 48 bits, on the FP32 pipe: k_panel_reg; in FP64 it took 0.9 ms per
// block on this GPU's FP64 units), the block row and column are solved in
// FP32 (k_trsm_reg),
// and the Schur update C22 -= L21 U12 runs on the tensor cores with BF16
// (split) or tile-scaled e4m3 operands and FP32 accumulation.
cudaError_t factor_tc(genp_factors *F, cudaStream_t s) {
    float *C = static_cast<float *>(F->C);
    const int64_t n = F->n, ldc = F->ldc;
    const int nb = (int)F->nb;
    const int terms = split_terms(F->prec);
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(k_trsm_reg<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)trsm_smem<float>(128));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_panel_reg<float, dfloat>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)panel_smem<dfloat>(128));
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    note_launch();
    k_maxabs<float><<<152 * 4, 256, 0, s>>>(C, n, ldc, &F->st->max_abs_c);
    for (int64_t k0 = 0; k0 < n; k0 += nb) {
        const int kb = (int)(n - k0 < nb ? n - k0 : nb);
        note_launch();
        k_panel_reg<float, dfloat><<<1, kPanelThreads, panel_smem<dfloat>(kb), s>>>(C, ldc, k0, kb, F->st);
        const int64_t rem = n - k0 - kb;
        if (rem <= 0) break;
        const TrsmRange rg{k0 + kb, n, k0 + kb, n};
        note_launch();
        k_trsm_reg<float, float><<<trsm_l_ctas(rg) + trsm_u_ctas(rg), kTrsmThreads, trsm_smem<float>(kb), s>>>(
            C, ldc, rg, k0, kb, F->st);
        float *L21 = C + (k0 + kb) * ldc + k0;
        float *U12 = C + k0 * ldc + k0 + kb;
        float *A22 = C + (k0 + kb) * ldc + k0 + kb;
        if (F->prec == GENP_FP8_E4M3) {
            // e4m3 operands, one power-of-two scale per 128 x 128 tile (kb <= 128:
            // a single k-tile, so each output tile takes one scale product)
            uint8_t *qa = reinterpret_cast<uint8_t *>(F->tcA), *qb = reinterpret_cast<uint8_t *>(F->tcB);
            const int64_t ldq = F->tc_ldq * 2;   // bytes
            float *sa = F->qscale, *sb = F->qscale + cdiv(n, 128);
            cudaError_t e = quant_e4m3<float>(L21, ldc, rem, kb, false, qa, ldq, sa, s);
            if (e == cudaSuccess) e = quant_e4m3<float>(U12, ldc, rem, kb, true, qb, ldq, sb, s);
            if (e == cudaSuccess)
                e = tc_gemm_e4m3(rem, rem, kb, -1.0f, qa, ldq, sa, qb, ldq, sb, 1.0f, A22, ldc, A22, ldc, s);
            if (e != cudaSuccess) return e;
            continue;
        }
        const int64_t Kq = (int64_t)kb * terms;
        cudaError_t e = split_rows<float>(L21, ldc, rem, kb, F->tcA, F->tc_ldq, terms, true, -1, s);
        if (e == cudaSuccess) e = split_cols_T<float>(U12, ldc, kb, rem, F->tcB, F->tc_ldq, terms, s);
        if (e == cudaSuccess)
            e = tc_gemm_bf16(rem, rem, Kq, -1.0f, F->tcA, F->tc_ldq, F->tcB, F->tc_ldq, 1.0f, A22, ldc, A22, ldc,
                             nullptr, s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// GENP_BF16_SLICED: blocked GENP in two levels on the double-float copy W
// of C.  The outer block column (2 nb wide) is factored by two inner steps of
// width nb: diagonal block and block row and column in double-float on the
// FP32 pipe, and the update of the second inner block (column and row) by
// the first on the tensor cores; the finished block column and block row are
// then rounded into C (exactly: a double-float value has 48 significant
// bits), and the outer Schur update W22 -= L21 U12 (K = 2 nb) runs on the
// tensor cores by exact digit slicing of the FP64 factors.  C ends up
// holding the factors.
cudaError_t factor_sliced(genp_factors *F, cudaStream_t s) {
    double *C = static_cast<double *>(F->C);
    dfloat *W = static_cast<dfloat *>(F->W);
    const int64_t n = F->n, ldc = F->ldc, ldw = F->ldw, ldq = F->tc_ldq;
    // outer steps of 512 (the tensor-core Schur updates' K: the largest at
    // which the digit-pair groups stay exact in FP32, so the fewest TMEM
    // read-outs per MMA), inner steps of nb
    const int nb = (int)F->nb, nbo = 2 * nb > kSlicedOuter ? 2 * nb : kSlicedOuter;
    // Look-ahead: each update that precedes a diagonal block first updates
    // that block's columns; the block is then factored on a second stream (one
    // SM, which the rest of the update leaves free) while the rest of the
    // update runs, and the block solves wait for both.
    // (the stream and events are made on the first factorization outside a
    // stream capture; a captured one joins the second stream into its graph)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        cap = cudaStreamCaptureStatusActive;
    }
    if (cap == cudaStreamCaptureStatusNone) {
        if (!F->la_stream && cudaStreamCreateWithFlags(&F->la_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            F->la_stream = nullptr;
        }
        for (auto &ev : F->la_ev)
            if (!ev && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                ev = nullptr;
            }
    }
    cudaStream_t s2 = F->la_stream;
    const bool ahead = s2 && F->la_ev[0] && F->la_ev[1];
    bool pending = false;   // the current block is being factored on s2
    auto block_ahead = [&](int64_t p0, int pb) -> cudaError_t {
        cudaError_t e = cudaEventRecord(F->la_ev[0], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s2, F->la_ev[0], 0);
        if (e == cudaSuccess) e = panel_only<dfloat, dfloat>(W, ldw, p0, pb, F->st, s2);
        if (e == cudaSuccess) e = cudaEventRecord(F->la_ev[1], s2);
        pending = e == cudaSuccess;
        return e;
    };
    // D[rows r0.., cols c0..c0+w) -= L U over the sliced operands' columns c0 - cb ..
    auto update = [&](int64_t m, int64_t w, int64_t kpad, int64_t bcol, dfloat *D) {
        return tc_gemm_sliced(F->nd, m, w, kpad, -1.0f, F->tcA, ldq, F->tcB + bcol * ldq, ldq, F->exps,
                              F->exps + n + bcol, D, ldw, s);
    };
    // the double-float copy and max |c_ij| in one pass over C
    cudaError_t e = df_from_f64(C, ldc, W, ldw, n, n, s, &F->st->max_abs_c);
    if (e != cudaSuccess) return e;
    for (int64_t k0 = 0; k0 < n; k0 += nbo) {
        const int kbo = (int)(n - k0 < nbo ? n - k0 : nbo);
        const int64_t e0 = k0 + kbo, remo = n - e0;
        for (int64_t i0 = k0; i0 < e0; i0 += nb) {
            const int kb = (int)(e0 - i0 < nb ? e0 - i0 : nb);
            const int64_t j0 = i0 + kb, rem = n - j0;
            if (pending) {
                e = cudaStreamWaitEvent(s, F->la_ev[1], 0);
                pending = false;
            } else {
                e = panel_only<dfloat, dfloat>(W, ldw, i0, kb, F->st, s);
            }
            // with the look-ahead, the block row beyond the next inner block is
            // solved later, while that block is factored: the path from one
            // diagonal block to the next takes only the block column and the
            // next block's columns of the block row
            const bool split = ahead && j0 < e0 && rem > 0;
            const int64_t nbn = split ? (e0 - j0 < nb ? e0 - j0 : nb) : 0;
            if (e == cudaSuccess)
                e = split ? trsm_range<dfloat, dfloat>(W, ldw, TrsmRange{j0, n, j0, j0 + nbn}, i0, kb, F->st, s)
                          : trsm_only<dfloat, dfloat>(W, ldw, n, i0, kb, F->st, s);
            if (e != cudaSuccess) return e;
            if (rem <= 0) break;
            if (j0 < e0) {
                // the rest of the outer block column, and its block row beyond it,
                // by the sliced product too: this inner step's L (rows j0..n) and U
                // (columns j0..n) are final, and are sliced once for both updates
                // straight from the double-float matrix (each entry exactly as
                // FP64; their FP64 copy in C is made at the end of the outer step)
                const int64_t w2 = e0 - j0;
                const int nb2 = (int)(w2 < nb ? w2 : nb);   // the next inner block
                const dfloat *Lw = W + j0 * ldw + i0;
                const dfloat *Uw = W + i0 * ldw + j0;
                unsigned long long *kk = reinterpret_cast<unsigned long long *>(F->exps + 2 * n);
                const int64_t kp = sliced_kpad(kb);
                e = sliced_inner_exps(Lw, ldw, rem, kb, kk, s);
                if (e == cudaSuccess) e = slice_rows(F->nd, Lw, ldw, rem, kb, F->tcA, ldq, F->exps, s, kk);
                if (split) {
                    if (e == cudaSuccess) e = slice_cols_T(F->nd, Uw, ldw, kb, nb2, F->tcB, ldq, F->exps + n, s, kk);
                    if (e == cudaSuccess) e = update(rem, nb2, kp, 0, W + j0 * ldw + j0);
                    if (e == cudaSuccess) e = block_ahead(j0, nb2);
                    const int prev = sliced_spare_sms(1);
                    // the rest of the block row, solved and sliced beside the next block
                    if (e == cudaSuccess)
                        e = trsm_range<dfloat, dfloat>(W, ldw, TrsmRange{j0, j0, j0 + nb2, n}, i0, kb, F->st, s);
                    if (e == cudaSuccess)
                        e = slice_cols_T(F->nd, Uw + nb2, ldw, kb, rem - nb2, F->tcB + nb2 * ldq, ldq,
                                         F->exps + n + nb2, s, kk);
                    if (e == cudaSuccess && w2 > nb2) e = update(rem, w2 - nb2, kp, nb2, W + j0 * ldw + j0 + nb2);
                    if (e == cudaSuccess && remo > 0) e = update(w2, remo, kp, w2, W + j0 * ldw + e0);
                    sliced_spare_sms(prev);
                } else {
                    if (e == cudaSuccess) e = slice_cols_T(F->nd, Uw, ldw, kb, rem, F->tcB, ldq, F->exps + n, s, kk);
                    if (e == cudaSuccess) e = update(rem, w2, kp, 0, W + j0 * ldw + j0);
                    if (e == cudaSuccess && remo > 0) e = update(w2, remo, kp, w2, W + j0 * ldw + e0);
                }
                if (e != cudaSuccess) return e;
            }
        }
        // this step's factors: block column (diagonal block included) and block row
        e = df_to_f64(W + k0 * ldw + k0, ldw, C + k0 * ldc + k0, ldc, n - k0, kbo, s);
        if (e == cudaSuccess && remo > 0) e = df_to_f64(W + k0 * ldw + e0, ldw, C + k0 * ldc + e0, ldc, kbo, remo, s);
        if (e != cudaSuccess) return e;
        if (remo <= 0) break;
        const double *L21 = C + e0 * ldc + k0;
        const double *U12 = C + k0 * ldc + e0;
        // GENP scales column k of L21 by 1/u_kk and row k of U12 with the
        // pivots: a power-of-two balance of the inner dimension (L21 D^-1,
        // D U12, exact) keeps each slicing row / column within a few binades
        // (the unrefined backward error drops about a thousandfold)
        unsigned long long *kexp = reinterpret_cast<unsigned long long *>(F->exps + 2 * n);
        e = sliced_inner_exps(L21, ldc, remo, kbo, kexp, s);
        if (e == cudaSuccess) e = slice_rows(F->nd, L21, ldc, remo, kbo, F->tcA, ldq, F->exps, s, kexp);
        if (e == cudaSuccess) e = slice_cols_T(F->nd, U12, ldc, kbo, remo, F->tcB, ldq, F->exps + n, s, kexp);
        const int64_t kp = sliced_kpad(kbo);
        const int nb2 = (int)(remo < nb ? remo : nb);       // the next step's first block
        if (ahead) {
            if (e == cudaSuccess) e = update(remo, nb2, kp, 0, W + e0 * ldw + e0);
            if (e == cudaSuccess) e = block_ahead(e0, nb2);
            const int prev = sliced_spare_sms(1);
            if (e == cudaSuccess && remo > nb2) e = update(remo, remo - nb2, kp, nb2, W + e0 * ldw + e0 + nb2);
            sliced_spare_sms(prev);
        } else if (e == cudaSuccess) {
            e = update(remo, remo, kp, 0, W + e0 * ldw + e0);
        }
        if (e != cudaSuccess) return e;
    }
    if (pending) {   // not reached (the last block is factored in place), kept for safety
        e = cudaStreamWaitEvent(s, F->la_ev[1], 0);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t maxabs_f64(const double *C, int64_t n, int64_t ldc, unsigned long long *out, cudaStream_t s) {
    note_launch();
    k_maxabs<double><<<152 * 4, 256, 0, s>>>(C, n, ldc, out);
    return cudaGetLastError();
}

cudaError_t status_reset(genp_factors *F, cudaStream_t s) {
    note_launch();
    k_status_reset<<<1, 1, 0, s>>>(F->st);
    return cudaGetLastError();
}

cudaError_t factor_run(genp_factors *F, cudaStream_t s) {
    cudaError_t e = status_reset(F, s);
    if (e != cudaSuccess) return e;
    switch (F->prec) {
        case GENP_FP64: e = F->block ? factor_block(F, s) : factor_typed<double, double>(F, s); break;
        case GENP_FP32: e = factor_typed<float, float>(F, s); break;
        case GENP_BF16:
        case GENP_BF16X3:
        case GENP_FP8_E4M3: e = factor_tc(F, s); break;
        case GENP_BF16_SLICED: e = factor_sliced(F, s); break;
        default: return cudaErrorNotSupported;
    }
    // the solves apply the diagonal blocks of L and U through their inverses
    // (block GE writes its pivot blocks' inverses itself)
    if (e == cudaSuccess && !F->block) e = invert_diag_blocks(F, s);
    return e;
}

}  // namespace genp
