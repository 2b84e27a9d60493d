// batched_escalate.cu -- the batched solve's fallback for systems whose
// FP32-factor refinement did not reach its target.
//
// A second persistent launch after the main batched kernel: each CTA pops
// systems from its own queue, skips those already solved, and for the rest
// forms C = A G again in double-float arithmetic (pairs of floats, about 48
// bits, on the FP32 pipe, which GB300 runs 64 times faster than FP64),
// factors it in its own scratch (blocked GENP: the diagonal block by the
// unblocked recurrence in shared memory, block row and column by
// substitution, Schur update by the CTA GEMM) and continues the FP64
// refinement of the system's current x by GMRES-IR with those factors as the
// preconditioner.  With no such system the launch only walks the queue.
#include "genp_internal.cuh"

#include <math.h>

#include "dfloat.cuh"

namespace genp {
namespace {

constexpr int BT = 256;     // threads per CTA
constexpr int TL = 64;      // CTA GEMM output tile
constexpr int KS = 16;      // CTA GEMM K step
constexpr int MAXNB = 64;   // largest factorization block
constexpr int SB = 32;      // solve block
constexpr int MAXRHS = 16;

template <typename T>
struct SmemGemm {
    T As[KS][TL];
    T Bs[KS][TL];
};
template <typename T>
struct SmemPanel {
    T a[MAXNB][MAXNB + 1];
    T x[TL][MAXNB + 1];
};
template <typename T>
struct SmemSolve {
    T t[SB][SB + 1];
    T y[SB][MAXRHS];
};
union Smem {
    SmemGemm<dfloat> gd;
    SmemPanel<dfloat> pd;
    SmemSolve<dfloat> sd;
};
template <typename T> __device__ __forceinline__ SmemGemm<T> &gemm_sm(Smem &s);
template <> __device__ __forceinline__ SmemGemm<dfloat> &gemm_sm<dfloat>(Smem &s) { return s.gd; }
template <typename T> __device__ __forceinline__ SmemPanel<T> &panel_sm(Smem &s);
template <> __device__ __forceinline__ SmemPanel<dfloat> &panel_sm<dfloat>(Smem &s) { return s.pd; }
template <typename T> __device__ __forceinline__ SmemSolve<T> &solve_sm(Smem &s);
template <> __device__ __forceinline__ SmemSolve<dfloat> &solve_sm<dfloat>(Smem &s) { return s.sd; }

struct SmemCtl {
    int idx;
    int done;
    int cmax_bits;
    unsigned long long rn[MAXRHS], xn[MAXRHS], bn[MAXRHS];
    unsigned long long anorm;
    double eta, eta_prev;
    float min_piv, max_piv, max_u;
    long long breakdown;
};

__device__ __forceinline__ float circ_at(const float *g, int64_t n, int64_t d) {
    d %= n;
    if (d < 0) d += n;
    return g[d];
}

__device__ __forceinline__ void smax_u64(unsigned long long *p, double v) {
    atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

// C = alpha * A * B + beta * C for one CTA in T arithmetic; B is dense (ldb)
// or, when g is non-null, the circulant B[k][j] = g[(k - j) mod gn].
template <typename TA, typename TB, typename T>
__device__ void cta_gemm(int m, int n, int k, T alpha, const TA *A, int64_t lda, const TB *B, int64_t ldb,
                         const float *g, int64_t gn, T beta, T *C, int64_t ldc, SmemGemm<T> &sm) {
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    for (int i0 = 0; i0 < m; i0 += TL)
        for (int j0 = 0; j0 < n; j0 += TL) {
            T acc[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
            for (int k0 = 0; k0 < k; k0 += KS) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int lin = tid + e * BT;
                    const int r = lin / KS, kk = lin % KS;
                    const int gr = i0 + r, gk = k0 + kk;
                    sm.As[kk][r] = (gr < m && gk < k) ? (T)A[(int64_t)gr * lda + gk] : T(0);
                    const int kk2 = lin / TL, c = lin % TL;
                    const int gk2 = k0 + kk2, gc = j0 + c;
                    T b = T(0);
                    if (gk2 < k && gc < n) b = g ? (T)circ_at(g, gn, (int64_t)gk2 - gc) : (T)B[(int64_t)gk2 * ldb + gc];
                    sm.Bs[kk2][c] = b;
                }
                __syncthreads();
#pragma unroll
                for (int kk = 0; kk < KS; ++kk) {
                    T a[4], b[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) a[i] = sm.As[kk][ty * 4 + i];
#pragma unroll
                    for (int j = 0; j < 4; ++j) b[j] = sm.Bs[kk][tx * 4 + j];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
                }
                __syncthreads();
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = i0 + ty * 4 + i;
                if (r >= m) continue;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int c = j0 + tx * 4 + j;
                    if (c >= n) continue;
                    T v = alpha * acc[i][j];
                    if (beta != T(0)) v = fma(beta, C[(int64_t)r * ldc + c], v);
                    C[(int64_t)r * ldc + c] = v;
                }
            }
        }
}

// Unblocked GENP of the kb x kb diagonal block at (k0, k0) in shared memory.
template <typename T>
__device__ void panel(T *C, int64_t ldc, int k0, int kb, SmemPanel<T> &p, SmemCtl &ctl) {
    const int tid = threadIdx.x;
    for (int idx = tid; idx < kb * kb; idx += BT) p.a[idx / kb][idx % kb] = C[(int64_t)(k0 + idx / kb) * ldc + k0 + idx % kb];
    __syncthreads();
    for (int k = 0; k < kb; ++k) {
        const T piv = p.a[k][k];
        if (tid == 0) {
            const float ap = (float)fabs((double)piv);
            if (!(ap > 0.f) || !isfinite(ap)) {
                if (ctl.breakdown < 0) ctl.breakdown = k0 + k;
            } else {
                ctl.min_piv = fminf(ctl.min_piv, ap);
                ctl.max_piv = fmaxf(ctl.max_piv, ap);
            }
        }
        for (int i = k + 1 + tid; i < kb; i += BT) p.a[i][k] = p.a[i][k] / piv;
        __syncthreads();
        const int rem = kb - k - 1;
        for (int idx = tid; idx < rem * rem; idx += BT) {
            const int i = k + 1 + idx / rem, j = k + 1 + idx % rem;
            p.a[i][j] = fma(-p.a[i][k], p.a[k][j], p.a[i][j]);
        }
        __syncthreads();
    }
    float um = 0.f;
    for (int idx = tid; idx < kb * kb; idx += BT) {
        const int i = idx / kb, j = idx % kb;
        C[(int64_t)(k0 + i) * ldc + k0 + j] = p.a[i][j];
        if (j >= i) um = fmaxf(um, (float)fabs((double)p.a[i][j]));
    }
    for (int o = 16; o > 0; o >>= 1) um = fmaxf(um, __shfl_xor_sync(0xffffffffu, um, o));
    if ((tid & 31) == 0) atomicMax((int *)&ctl.max_u, __float_as_int(um));
    __syncthreads();
}

// U12 = L11^{-1} C12 by forward substitution (L11 unit lower in p.a), in
// place, chunks of TL columns; tracks max |U12| in um.
template <typename T>
__device__ void trsm_left(T *C, int64_t ldc, int k0, int kb, int c0, int n, SmemPanel<T> &p, float &um) {
    const int tid = threadIdx.x;
    for (int cc = c0; cc < n; cc += TL) {
        const int w = min(TL, n - cc);
        for (int idx = tid; idx < kb * w; idx += BT) p.x[idx % w][idx / w] = C[(int64_t)(k0 + idx / w) * ldc + cc + idx % w];
        __syncthreads();
        for (int k = 0; k + 1 < kb; ++k) {
            const int rem = kb - k - 1;
            for (int idx = tid; idx < rem * w; idx += BT) {
                const int r = k + 1 + idx / w, c = idx % w;
                p.x[c][r] = fma(-p.a[r][k], p.x[c][k], p.x[c][r]);
            }
            __syncthreads();
        }
        for (int idx = tid; idx < kb * w; idx += BT) {
            const T v = p.x[idx % w][idx / w];
            C[(int64_t)(k0 + idx / w) * ldc + cc + idx % w] = v;
            um = fmaxf(um, (float)fabs((double)v));
        }
        __syncthreads();
    }
}

// L21 = C21 U11^{-1} by substitution along each row (U11 upper in p.a), in
// place, chunks of TL rows.
template <typename T>
__device__ void trsm_right(T *C, int64_t ldc, int k0, int kb, int r0, int n, SmemPanel<T> &p) {
    const int tid = threadIdx.x;
    for (int rr = r0; rr < n; rr += TL) {
        const int h = min(TL, n - rr);
        for (int idx = tid; idx < h * kb; idx += BT) p.x[idx / kb][idx % kb] = C[(int64_t)(rr + idx / kb) * ldc + k0 + idx % kb];
        __syncthreads();
        for (int j = 0; j < kb; ++j) {
            for (int r = tid; r < h; r += BT) p.x[r][j] = p.x[r][j] / p.a[j][j];
            __syncthreads();
            const int rem = kb - j - 1;
            for (int idx = tid; idx < h * rem; idx += BT) {
                const int r = idx / rem, l = j + 1 + idx % rem;
                p.x[r][l] = fma(-p.x[r][j], p.a[j][l], p.x[r][l]);
            }
            __syncthreads();
        }
        for (int idx = tid; idx < h * kb; idx += BT) C[(int64_t)(rr + idx / kb) * ldc + k0 + idx % kb] = p.x[idx / kb][idx % kb];
        __syncthreads();
    }
}

template <typename T>
__device__ void factor_sys(T *C, int n, int nb, Smem &sm, SmemCtl &ctl) {
    float um = 0.f;
    for (int k0 = 0; k0 < n; k0 += nb) {
        const int kb = min(nb, n - k0);
        panel<T>(C, n, k0, kb, panel_sm<T>(sm), ctl);
        const int rem = n - k0 - kb;
        if (rem <= 0) break;
        trsm_left<T>(C, n, k0, kb, k0 + kb, n, panel_sm<T>(sm), um);
        trsm_right<T>(C, n, k0, kb, k0 + kb, n, panel_sm<T>(sm));
        cta_gemm<T, T, T>(rem, rem, kb, T(-1), C + (int64_t)(k0 + kb) * n + k0, n, C + (int64_t)k0 * n + k0 + kb, n,
                          nullptr, 0, T(1), C + (int64_t)(k0 + kb) * n + k0 + kb, n, gemm_sm<T>(sm));
        __syncthreads();
    }
    for (int o = 16; o > 0; o >>= 1) um = fmaxf(um, __shfl_xor_sync(0xffffffffu, um, o));
    if ((threadIdx.x & 31) == 0) atomicMax((int *)&ctl.max_u, __float_as_int(um));
    __syncthreads();
}

// Y <- op^{-1} Y for the factors in C (n x n), Y n x nr (ld nr), blocked by SB.
// trans = false: U^{-1} L^{-1} Y.  trans = true: L^{-T} U^{-T} Y.
template <typename T>
__device__ void solve_sys(const T *C, int n, T *Y, int nr, bool trans, SmemSolve<T> &s) {
    const int tid = threadIdx.x;
    const int nblk = (n + SB - 1) / SB;
    for (int pass = 0; pass < 2; ++pass) {
        // pass 0: forward (L, or U^T); pass 1: backward (U, or L^T)
        const bool unit = trans ? (pass == 1) : (pass == 0);
        for (int q = 0; q < nblk; ++q) {
            const int blk = pass == 0 ? q : nblk - 1 - q;
            const int b0 = blk * SB, bs = min(SB, n - b0);
            for (int idx = tid; idx < bs * bs; idx += BT) {
                const int i = idx / bs, j = idx % bs;
                s.t[i][j] = trans ? C[(int64_t)(b0 + j) * n + b0 + i] : C[(int64_t)(b0 + i) * n + b0 + j];
            }
            for (int idx = tid; idx < bs * nr; idx += BT) s.y[idx / nr][idx % nr] = Y[(int64_t)(b0 + idx / nr) * nr + idx % nr];
            __syncthreads();
            for (int st = 0; st < bs; ++st) {
                const int k = pass == 0 ? st : bs - 1 - st;
                if (!unit) {
                    if (tid < nr) s.y[k][tid] = s.y[k][tid] / s.t[k][k];
                    __syncthreads();
                }
                const int lo = pass == 0 ? k + 1 : 0, hi = pass == 0 ? bs : k;
                for (int idx = tid; idx < (hi - lo) * nr; idx += BT) {
                    const int i = lo + idx / nr, c = idx % nr;
                    s.y[i][c] = fma(-s.t[i][k], s.y[k][c], s.y[i][c]);
                }
                __syncthreads();
            }
            for (int idx = tid; idx < bs * nr; idx += BT) Y[(int64_t)(b0 + idx / nr) * nr + idx % nr] = s.y[idx / nr][idx % nr];
            // update the rows not yet solved with this block's values
            const int r_lo = pass == 0 ? b0 + bs : 0, r_hi = pass == 0 ? n : b0;
            for (int i = r_lo + tid; i < r_hi; i += BT) {
                T acc[MAXRHS];
                for (int c = 0; c < nr; ++c) acc[c] = T(0);
                for (int k = 0; k < bs; ++k) {
                    const T l = trans ? C[(int64_t)(b0 + k) * n + i] : C[(int64_t)i * n + b0 + k];
                    for (int c = 0; c < nr; ++c) acc[c] = fma(l, s.y[k][c], acc[c]);
                }
                for (int c = 0; c < nr; ++c) Y[(int64_t)i * nr + c] -= acc[c];
            }
            __syncthreads();
        }
    }
}

// R = B - A X (FP64), column norms into ctl; ||A||_inf too when `anorm`.
template <typename TA>
__device__ void residual(const TA *A, int n, const double *B, const double *X, double *R, int nr, bool anorm,
                         SmemCtl &ctl) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < n; i += BT / 32) {
        double acc[MAXRHS];
        for (int c = 0; c < nr; ++c) acc[c] = 0.0;
        double rs = 0.0;
        for (int j = lane; j < n; j += 32) {
            const double a = (double)A[(int64_t)i * n + j];
            rs += fabs(a);
            for (int c = 0; c < nr; ++c) acc[c] = fma(a, X[(int64_t)j * nr + c], acc[c]);
        }
        for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
        if (anorm && lane == 0) smax_u64(&ctl.anorm, rs);
        for (int c = 0; c < nr; ++c) {
            double v = acc[c];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) {
                const double r = B[(int64_t)i * nr + c] - v;
                R[(int64_t)i * nr + c] = r;
                smax_u64(&ctl.rn[c], fabs(r));
                smax_u64(&ctl.xn[c], fabs(X[(int64_t)i * nr + c]));
                smax_u64(&ctl.bn[c], fabs(B[(int64_t)i * nr + c]));
            }
        }
    }
}

// ---------------------------------------------------------------------------
// GMRES-IR for the escalated systems (Carson & Higham 2018): the outer step
// takes r = b - A x in FP64 and solves C d = r by FP64 GMRES on the
// left-preconditioned system U^-1 L^-1 C d = U^-1 L^-1 r with the
// double-float factors (C v applied as A (G v) in double-float), then
// x += G d in FP64.  Classic refinement needs u_df kappa(C) growth < 1, which the
// systems that reach this launch (kappa(A G) up to ~1e10) can miss; GMRES
// needs the factors only as a preconditioner.
// ---------------------------------------------------------------------------
constexpr int KRY = 20;   // Krylov vectors per outer step and right-hand side
constexpr int NG = 4;     // right-hand sides iterated in lockstep

struct GmresCtl {
    double H[NG][KRY + 1][KRY];
    double cs[NG][KRY], sn[NG][KRY], gv[NG][KRY + 1], y[NG][KRY];
    double beta[NG];
    double red[BT / 32][NG];
    double val[NG];
    int kend[NG];
    int active;
};

// Sums over the CTA of the per-thread values v[0 .. w-1]; every thread gets
// the totals in gc.val.
__device__ void cta_sums(double (&v)[NG], int w, GmresCtl &gc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < NG; ++c)
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < NG; ++c) gc.red[warp][c] = v[c];
    __syncthreads();
    if (threadIdx.x < w) {
        double t = 0.0;
        for (int q = 0; q < BT / 32; ++q) t += gc.red[q][threadIdx.x];
        gc.val[threadIdx.x] = t;
    }
    __syncthreads();
}

// The Krylov operator's products in double-float (about 2^-44 per
// operation, on the FP32 pipe, which GB300 runs 64 times faster than FP64):
// the inner solve only has to be accurate enough to contract the FP64
// residual of the outer step.  One warp per row, w <= NG columns of v
// (ld NG) into out (ld NG).
__device__ void g_apply_df(const float *G, const float *g, int n, const double *v, double *out, int w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < n; i += BT / 32) {
        dfloat acc[NG];
#pragma unroll
        for (int c = 0; c < NG; ++c) acc[c] = dfloat(0.0f);
        for (int j = lane; j < n; j += 32) {
            const dfloat gij(g ? circ_at(g, n, (int64_t)i - j) : G[(int64_t)i * n + j]);
#pragma unroll
            for (int c = 0; c < NG; ++c)
                if (c < w) acc[c] = acc[c] + gij * dfloat(v[(int64_t)j * NG + c]);
        }
#pragma unroll
        for (int c = 0; c < NG; ++c)
            for (int o = 16; o > 0; o >>= 1) {
                dfloat t;
                t.hi = __shfl_xor_sync(0xffffffffu, acc[c].hi, o);
                t.lo = __shfl_xor_sync(0xffffffffu, acc[c].lo, o);
                acc[c] = acc[c] + t;
            }
        if (lane < w) {
            dfloat r = acc[0];
#pragma unroll
            for (int c = 1; c < NG; ++c) r = c == lane ? acc[c] : r;
            out[(int64_t)i * NG + lane] = (double)r;
        }
    }
}

template <typename TA>
__device__ void a_apply_df(const TA *A, int n, const double *v, double *out, int w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < n; i += BT / 32) {
        dfloat acc[NG];
#pragma unroll
        for (int c = 0; c < NG; ++c) acc[c] = dfloat(0.0f);
        for (int j = lane; j < n; j += 32) {
            const dfloat aij((double)A[(int64_t)i * n + j]);
#pragma unroll
            for (int c = 0; c < NG; ++c)
                if (c < w) acc[c] = acc[c] + aij * dfloat(v[(int64_t)j * NG + c]);
        }
#pragma unroll
        for (int c = 0; c < NG; ++c)
            for (int o = 16; o > 0; o >>= 1) {
                dfloat t;
                t.hi = __shfl_xor_sync(0xffffffffu, acc[c].hi, o);
                t.lo = __shfl_xor_sync(0xffffffffu, acc[c].lo, o);
                acc[c] = acc[c] + t;
            }
        if (lane < w) {
            dfloat r = acc[0];
#pragma unroll
            for (int c = 1; c < NG; ++c) r = c == lane ? acc[c] : r;
            out[(int64_t)i * NG + lane] = (double)r;
        }
    }
}

// W <- U^-1 L^-1 W (n x w, ld NG) with the double-float factors, through Yd
__device__ void precond(const dfloat *Cf, int n, double *W, int w, dfloat *Yd, Smem &sm) {
    for (int e = threadIdx.x; e < n * w; e += BT) Yd[e] = dfloat(W[(int64_t)(e / w) * NG + e % w]);
    __syncthreads();
    solve_sys<dfloat>(Cf, n, Yd, w, false, solve_sm<dfloat>(sm));
    __syncthreads();
    for (int e = threadIdx.x; e < n * w; e += BT) W[(int64_t)(e / w) * NG + e % w] = (double)Yd[e];
    __syncthreads();
}

// GMRES on C d = r for the columns c0 .. c0 + w - 1 of R (ld nr) in
// lockstep (one preconditioner solve and one pass over G and A per Krylov
// step for all of them), each with its own basis, Hessenberg matrix and
// stopping point; then x += G d in FP64.  V holds (KRY + 1) n NG doubles,
// T two n x NG work blocks.
template <typename TA>
__device__ void gmres_group(const TA *A, const dfloat *Cf, const float *G, const float *g, const double *R, int nr,
                            int c0, int w, double *X, double *V, double *T, dfloat *Yd, int n, Smem &sm,
                            GmresCtl &gc) {
    const int tid = threadIdx.x;
    double *W = T, *Tm = T + (int64_t)n * NG;
    for (int e = tid; e < n * NG; e += BT) {
        const int i = e / NG, c = e % NG;
        W[e] = c < w ? R[(int64_t)i * nr + c0 + c] : 0.0;
    }
    __syncthreads();
    precond(Cf, n, W, w, Yd, sm);
    double part[NG];
#pragma unroll
    for (int c = 0; c < NG; ++c) part[c] = 0.0;
    for (int e = tid; e < n * NG; e += BT) part[e % NG] += W[e] * W[e];   // BT is a multiple of NG
    cta_sums(part, w, gc);
    if (tid < NG) {
        const double b = tid < w ? sqrt(gc.val[tid]) : 0.0;
        gc.beta[tid] = (b > 0.0 && isfinite(b)) ? b : 0.0;
        gc.gv[tid][0] = gc.beta[tid];
        gc.kend[tid] = 0;
    }
    if (tid == 0) gc.active = 0;
    __syncthreads();
    if (tid < w && gc.beta[tid] > 0.0) atomicOr(&gc.active, 1 << tid);
    __syncthreads();
    if (!gc.active) return;
    for (int e = tid; e < n * NG; e += BT) {
        const double b = gc.beta[e % NG];
        V[e] = b > 0.0 ? W[e] / b : 0.0;
    }
    __syncthreads();
    for (int k = 0; k < KRY && gc.active; ++k) {
        const double *vk = V + (int64_t)k * n * NG;
        g_apply_df(G, g, n, vk, Tm, w);
        __syncthreads();
        a_apply_df<TA>(A, n, Tm, W, w);
        __syncthreads();
        precond(Cf, n, W, w, Yd, sm);
        // modified Gram-Schmidt, all columns at once
        for (int i = 0; i <= k; ++i) {
            const double *vi = V + (int64_t)i * n * NG;
#pragma unroll
            for (int c = 0; c < NG; ++c) part[c] = 0.0;
            for (int e = tid; e < n * NG; e += BT) part[e % NG] += W[e] * vi[e];
            cta_sums(part, w, gc);
            for (int e = tid; e < n * NG; e += BT) W[e] -= gc.val[e % NG] * vi[e];
            if (tid < w) gc.H[tid][i][k] = gc.val[tid];
            __syncthreads();
        }
#pragma unroll
        for (int c = 0; c < NG; ++c) part[c] = 0.0;
        for (int e = tid; e < n * NG; e += BT) part[e % NG] += W[e] * W[e];
        cta_sums(part, w, gc);
        double *vn = V + (int64_t)(k + 1) * n * NG;
        for (int e = tid; e < n * NG; e += BT) {
            const double hk = sqrt(gc.val[e % NG]);
            vn[e] = hk > 0.0 ? W[e] / hk : 0.0;
        }
        if (tid < w && ((gc.active >> tid) & 1)) {
            // this column's Givens rotations: the earlier ones on the new
            // column of H, then a new one
            const int c = tid;
            const double hk = sqrt(gc.val[c]);
            for (int i = 0; i < k; ++i) {
                const double a = gc.H[c][i][k], b = gc.H[c][i + 1][k];
                gc.H[c][i][k] = gc.cs[c][i] * a + gc.sn[c][i] * b;
                gc.H[c][i + 1][k] = -gc.sn[c][i] * a + gc.cs[c][i] * b;
            }
            const double a = gc.H[c][k][k];
            const double r = hypot(a, hk);
            gc.cs[c][k] = r > 0.0 ? a / r : 1.0;
            gc.sn[c][k] = r > 0.0 ? hk / r : 0.0;
            gc.H[c][k][k] = r;
            gc.gv[c][k + 1] = -gc.sn[c][k] * gc.gv[c][k];
            gc.gv[c][k] = gc.cs[c][k] * gc.gv[c][k];
            gc.kend[c] = k + 1;
            // converged (or a lucky breakdown): this column stops here
            if (!(fabs(gc.gv[c][k + 1]) > 1e-12 * gc.beta[c]) || !(hk > 0.0)) atomicAnd(&gc.active, ~(1 << c));
        }
        __syncthreads();
    }
    if (tid < w) {   // back substitution for each column's y
        const int c = tid, m = gc.kend[c];
        for (int i = m - 1; i >= 0; --i) {
            double sacc = gc.gv[c][i];
            for (int j = i + 1; j < m; ++j) sacc -= gc.H[c][i][j] * gc.y[c][j];
            gc.y[c][i] = gc.H[c][i][i] != 0.0 ? sacc / gc.H[c][i][i] : 0.0;
        }
    }
    __syncthreads();
    for (int e = tid; e < n * NG; e += BT) {
        const int c = e % NG;
        double d = 0.0;
        if (c < w)
            for (int i = 0; i < gc.kend[c]; ++i) d += gc.y[c][i] * V[(int64_t)i * n * NG + e];
        W[e] = d;
    }
    __syncthreads();
    // x += G d, FP64
    const int lane = tid & 31, warp = tid >> 5;
    for (int i = warp; i < n; i += BT / 32) {
        double acc[NG];
#pragma unroll
        for (int c = 0; c < NG; ++c) acc[c] = 0.0;
        for (int j = lane; j < n; j += 32) {
            const double gij = g ? (double)circ_at(g, n, (int64_t)i - j) : (double)G[(int64_t)i * n + j];
#pragma unroll
            for (int c = 0; c < NG; ++c) acc[c] = fma(gij, W[(int64_t)j * NG + c], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < NG; ++c) {
            for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
            if (lane == 0 && c < w) X[(int64_t)i * nr + c0 + c] += acc[c];
        }
    }
    __syncthreads();
}

// GMRES-IR outer loop: stop at eta <= tol, when eta fails to halve, or
// after max_iter steps.  Returns the steps taken.
template <typename TA>
__device__ int refine_gmres(const TA *A, const dfloat *Cf, const float *G, const float *g, const double *B,
                            double *X, double *R, double *V, double *T, dfloat *Yd, int n, int nr, int max_iter,
                            double tol, double &eta0, double &eta, Smem &sm, SmemCtl &ctl, GmresCtl &gc) {
    const int tid = threadIdx.x;
    int it = 0;
    if (tid == 0) ctl.eta_prev = INFINITY;
    for (;; ++it) {
        if (tid < MAXRHS) ctl.rn[tid] = ctl.xn[tid] = ctl.bn[tid] = 0ull;
        __syncthreads();
        residual<TA>(A, n, B, X, R, nr, it == 0, ctl);
        __syncthreads();
        if (tid == 0) {
            const double an = __longlong_as_double((long long)ctl.anorm);
            double e = 0.0;
            for (int c = 0; c < nr; ++c) {
                double v = __longlong_as_double((long long)ctl.rn[c]) /
                           (an * __longlong_as_double((long long)ctl.xn[c]) + __longlong_as_double((long long)ctl.bn[c]));
                if (!(v == v)) v = INFINITY;
                e = fmax(e, v);
            }
            ctl.eta = e;
            ctl.done = (e <= tol) || (it > 0 && e > 0.5 * ctl.eta_prev) || it >= max_iter;
            ctl.eta_prev = e;
        }
        __syncthreads();
        eta = ctl.eta;
        if (it == 0) eta0 = eta;
        if (ctl.done) break;
        for (int c0 = 0; c0 < nr; c0 += NG)
            gmres_group<TA>(A, Cf, G, g, R, nr, c0, min(NG, nr - c0), X, V, T, Yd, n, sm, gc);
    }
    return it;
}

template <typename TA>
__global__ void __launch_bounds__(BT) k_batched_escalate(const BatchDesc *d, int count, int *counter,
                                                         const TA *Apool, const double *Bpool, double *Xpool,
                                                         const float *Gpool, const float *gpool, double *Rpool,
                                                         double *scratch64, int64_t stride, int nr, int circ,
                                                         int max_iter, double tol, BatchStatus *stat) {
    extern __shared__ __align__(16) unsigned char smraw[];
    Smem &sm = *reinterpret_cast<Smem *>(smraw);
    __shared__ SmemCtl ctl;
    __shared__ GmresCtl gc;
    const int tid = threadIdx.x;
    while (true) {
        if (tid == 0) ctl.idx = atomicAdd(counter, 1);
        __syncthreads();
        const int idx = ctl.idx;
        if (idx >= count) break;
        if (stat[idx].status == GENP_OK) {
            __syncthreads();
            continue;
        }
        const BatchDesc q = d[idx];
        const int n = (int)q.n;
        if (tid == 0) {
            ctl.breakdown = -1;
            ctl.min_piv = INFINITY;
            ctl.max_piv = 0.f;
            ctl.max_u = 0.f;
            ctl.anorm = 0ull;
        }
        __syncthreads();
        const TA *A = Apool + q.mat_off;
        const float *G = circ ? nullptr : Gpool + q.mat_off;
        const float *g = circ ? gpool + q.g_off : nullptr;
        const double *B = Bpool + q.vec_off;
        double *X = Xpool + q.vec_off;
        double *R = Rpool + q.vec_off;
        if (!(stat[idx].eta < INFINITY))   // no usable iterate: start from x = 0
            for (int e = tid; e < n * nr; e += BT) X[e] = 0.0;
        __syncthreads();
        double *base = scratch64 + (int64_t)blockIdx.x * stride;
        dfloat *Cd = reinterpret_cast<dfloat *>(base);                                         // n x n
        dfloat *Yd = Cd + 1024ll * 1024ll;                                                     // n x nr
        double *V = base + 1024ll * 1024ll + 1024ll * MAXRHS;                                 // (KRY + 1) x n x NG
        double *T = V + (int64_t)(KRY + 1) * 1024 * NG;                                        // 2 x n x NG
        cta_gemm<TA, float, dfloat>(n, n, n, dfloat(1), A, n, G, n, g, n, dfloat(0), Cd, n, sm.gd);
        __syncthreads();
        factor_sys<dfloat>(Cd, n, 32, sm, ctl);
        double e0 = 0.0, eta = INFINITY;
        const int it = refine_gmres<TA>(A, Cd, G, g, B, X, R, V, T, Yd, n, nr, max_iter, tol, e0, eta, sm, ctl, gc);
        if (tid == 0) {
            BatchStatus st = stat[idx];
            st.refine_iters += 1 + it;
            st.status = ctl.breakdown >= 0 ? GENP_ERR_BREAKDOWN : (eta <= tol ? GENP_OK : GENP_ERR_NOCONV);
            st.escalated = 2;
            st.eta = eta;
            stat[idx] = st;
        }
        __syncthreads();
    }
}

}  // namespace

// 8-byte elements of the per-CTA scratch (C as double-float: n^2 for
// n <= 1024; Y: n x 16 follows it, then the KRY + 1 Krylov blocks and two
// work blocks of n x NG doubles).
int64_t batched_escalate_stride() { return 1024ll * 1024ll + 1024ll * MAXRHS + (KRY + 3) * 1024ll * NG; }

int batched_escalate_blocks_per_sm() {
    int b = 1;
    cudaFuncSetAttribute(k_batched_escalate<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
    cudaFuncSetAttribute(k_batched_escalate<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batched_escalate<double>, BT, sizeof(Smem)) != cudaSuccess) {
        cudaGetLastError();
        b = 1;
    }
    return b < 1 ? 1 : b;
}

cudaError_t launch_batched_escalate(const BatchDesc *d, int count, int *counter, const void *Apool, bool a_f64,
                                    const double *Bpool, double *Xpool, const float *Gpool, const float *gpool,
                                    double *Rpool, double *scratch64, int nr, bool circ, int max_iter, double tol,
                                    BatchStatus *stat, int grid, cudaStream_t s) {
    const int64_t stride = batched_escalate_stride();
    note_launch();
    if (a_f64)
        k_batched_escalate<double><<<grid, BT, sizeof(Smem), s>>>(d, count, counter, (const double *)Apool, Bpool,
                                                                   Xpool, Gpool, gpool, Rpool, scratch64, stride, nr,
                                                                   circ ? 1 : 0, max_iter, tol, stat);
    else
        k_batched_escalate<float><<<grid, BT, sizeof(Smem), s>>>(d, count, counter, (const float *)Apool, Bpool,
                                                                  Xpool, Gpool, gpool, Rpool, scratch64, stride, nr,
                                                                  circ ? 1 : 0, max_iter, tol, stat);
    return cudaGetLastError();
}

}  // namespace genp
