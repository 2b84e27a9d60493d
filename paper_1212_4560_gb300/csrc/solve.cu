// solve.cu -- triangular solves with the GENP factors, refinement control
// and the adjoint's outer product.
//
// Each triangular solve is one persistent launch (k_trsv below), 16
// right-hand sides at a time.  The transposed pair (U^T then L^T) serves the
// adjoint (A^{-T} = L^{-T} U^{-T} G^T).  The 64 x 64 diagonal blocks of L and
// U are inverted once after every factorization (k_trtri_diag) and applied
// as small matrix-vector products, which keeps the solve's critical path (one
// diagonal block after another) short; GPU triangular-solve libraries do the
// same (e.g. MAGMA's trtri_diag + gemv).
//
// Refinement (Sec. 7.1) is steered on the device: every iteration's kernels
// read a `done` flag that the stopping test sets, so a whole refinement is
// enqueued at once with no host synchronization.
#include "genp_internal.cuh"
#include "dfloat.cuh"

#include <math.h>

namespace genp {
namespace {

constexpr int kTrsvMaxRhs = 16;   // right-hand sides per triangular-solve launch

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
    st->krylov_steps = 0;
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

// dA[i][j] = - sum_c Lam[i][c] X[j][c] as a streaming write (nrhs <= NR): a
// CTA covers 32 rows and 1024 columns, each thread 4 adjacent columns whose
// X rows it keeps in registers, and every row goes out as one contiguous
// 1 KiB (FP64) store per warp.  vec: 16-byte aligned rows (ldda % 4 == 0,
// aligned base), so the 4 values go out as 16- or 32-byte vector stores.
template <typename TD, int NR>
__global__ void __launch_bounds__(256) k_outer_rows(const double *Lam, int64_t ldl, const double *X, int64_t ldx,
                                                    int64_t n, int nrhs, TD *dA, int64_t ldda, int vec) {
    __shared__ double sl[32][NR];
    const int64_t i0 = (int64_t)blockIdx.y * 32;
    const int64_t j = ((int64_t)blockIdx.x * 256 + threadIdx.x) * 4;
    for (int idx = threadIdx.x; idx < 32 * NR; idx += 256) {
        const int r = idx / NR, c = idx % NR;
        sl[r][c] = (i0 + r < n && c < nrhs) ? Lam[(i0 + r) * ldl + c] : 0.0;
    }
    double xr[4][NR];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < NR; ++c) xr[q][c] = (j + q < n && c < nrhs) ? X[(j + q) * ldx + c] : 0.0;
    __syncthreads();
    if (j >= n) return;
    const bool full = vec && j + 3 < n;
    for (int r = 0; r < 32; ++r) {
        const int64_t i = i0 + r;
        if (i >= n) break;
        double v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            double acc = 0.0;
#pragma unroll
            for (int c = 0; c < NR; ++c) acc = fma(sl[r][c], xr[q][c], acc);
            v[q] = -acc;
        }
        TD *row = dA + i * ldda + j;
        if (full) {
            if constexpr (sizeof(TD) == 8) {
                reinterpret_cast<double2 *>(row)[0] = make_double2(v[0], v[1]);
                reinterpret_cast<double2 *>(row)[1] = make_double2(v[2], v[3]);
            } else {
                *reinterpret_cast<float4 *>(row) = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (j + q < n) row[q] = (TD)v[q];
        }
    }
}

// ---------------------------------------------------------------------------
// Triangular solves op(T) Y = Y in one persistent launch.  T is cut into
// 64 x 64 tiles and the diagonal blocks are taken one after the other (block
// j(q) at step q: j = q forward, nblk-1-q backward).  The CTA that draws
// ticket 0 walks the diagonal: for each block it applies the precomputed
// inverse of the diagonal tile plus one refinement step, publishes y_j, and
// subtracts op(T)[next][j] y_j from the next block itself, so the chain from
// one block to the next never waits on another CTA.  Every other ticket is a
// work item that sums op(T)[i][j(p)] y_j(p) over up to kSeg earlier steps p
// for one block i = j(q) two or more steps ahead, in registers, and
// subtracts the sum from Y_i with one set of FP64 (or FP32) atomics; a
// per-block counter, raised by the number of steps summed, tells the walker
// when all of block i's contributions have landed.  Items are handed out in
// the order the walker needs them (by target step q, then by p), each waits
// only for the y_j(p) it multiplies (all published before the walker reaches
// step q - 1), and the walker waits only for items of its current step,
// which hold smaller tickets than anything still waiting, so the launch
// cannot deadlock (it needs two or more CTAs).  Every wait is bounded: on
// timeout the kernel sets a device flag (read by genp_device_check) and goes
// on.
// ---------------------------------------------------------------------------
constexpr int TB = 64;          // tile
constexpr int kSeg = 16;        // tiles per work item
constexpr int kTrsvThreads = 256;
constexpr long long kSpinTicks = 4000000000LL;   // ~2 s at 2 GHz

__device__ int g_solve_timeout;

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Publishes a flag for the writes the whole CTA made before a __syncthreads:
// the barrier orders them before this thread's fence, and the fence and the
// release store (both GPU scope, cumulative) make them visible to any thread
// that reads the flag with acquire semantics.
__device__ __forceinline__ void publish(int *p) {
    __threadfence();
    st_release(p, 1);
}
__device__ bool wait_geq(const int *p, int target) {
    const long long t0 = clock64();
    while (ld_acquire(p) < target) {
        if (clock64() - t0 > kSpinTicks) return false;
        __nanosleep(64);
    }
    return true;
}
// work items of target step q >= 2: the q - 1 earlier steps p <= q - 2, kSeg per item
__device__ __forceinline__ int nchunks(int q) { return q < 2 ? 0 : (q - 1 + kSeg - 1) / kSeg; }
__device__ __forceinline__ double ldcg(const double *p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg(const float *p) { return __ldcg(p); }

template <typename T, int NR>
struct TrsvSmem {
    T S[TB][TB + 1];    // op(T_jj)^{-1} (walker) or the current tile (items)
    T D[TB][TB + 1];    // op(T_jj), its triangle only (walker)
    T O[TB][TB + 1];    // op(T)[next][j] (walker)
    T y[TB][NR];        // y_j
    T acc[TB][NR];      // right-hand side of the diagonal block, then its residual
    T carry[TB][NR];    // the walker's own contribution to the next block
};

// The walker's shared memory when it runs in double-float (factors held as
// double-float pairs, GENP_BF16_SLICED): the three tiles as hi / lo FP32
// planes with a row stride of 68, read with the quarters interleaved along k
// (quarter q takes k = q + 4 kk), so the 32 lanes of a warp (8 rows x 4
// quarters) hit 32 different banks; the vectors as double-float pairs.
constexpr int kDdLd = 68;
template <int NR>
struct TrsvSmemDD {
    float Sh[TB][kDdLd], Sl[TB][kDdLd];
    float Dh[TB][kDdLd], Dl[TB][kDdLd];
    float Oh[TB][kDdLd], Ol[TB][kDdLd];
    dfloat y[TB][NR], acc[TB][NR], carry[TB][NR];
};

// s + t += (ah + al)(v.hi + v.lo): TwoSum of the leading terms, the rounding
// error of the leading product (by FMA) and the cross terms gathered in t
// (Dekker 1971; Ogita, Rump & Oishi 2005).
__device__ __forceinline__ void dd_mac(float &s, float &t, float ah, float al, dfloat v) {
    const float p = ah * v.hi;
    const float pe = fmaf(ah, v.hi, -p);
    const float cross = fmaf(ah, v.lo, al * v.hi);
    const float sn = s + p, bb = sn - s;
    const float err = (s - (sn - bb)) + (p - bb);
    s = sn;
    t += err + (pe + cross);
}

// part[c] = sum_k M[r][k] V[k][c] in double-float, summed over the 4 quarter
// threads of row r (thread = 4 r + quarter)
template <int NR>
__device__ __forceinline__ void tile_gemv_dd(const float (*Mh)[kDdLd], const float (*Ml)[kDdLd], const dfloat (*V)[NR],
                                             int r, int qq, dfloat (&part)[NR]) {
    float s[NR], t[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) s[c] = t[c] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
        const int k = qq + 4 * kk;
        const float ah = Mh[r][k], al = Ml[r][k];
#pragma unroll
        for (int c = 0; c < NR; ++c) dd_mac(s[c], t[c], ah, al, V[k][c]);
    }
#pragma unroll
    for (int c = 0; c < NR; ++c) {
        dfloat a = df_norm(s[c], t[c]);
        for (int o = 1; o <= 2; o <<= 1) {
            dfloat b;
            b.hi = __shfl_xor_sync(0xffffffffu, a.hi, o);
            b.lo = __shfl_xor_sync(0xffffffffu, a.lo, o);
            a = a + b;
        }
        part[c] = a;
    }
}

// part[c] += sum over this thread's quarter of k of M[r][k] V[k][c] (thread = 4 r + quarter)
template <typename T, int NR>
__device__ __forceinline__ void tile_gemv_acc(const T (*M)[TB + 1], const T (*V)[NR], int r, int qq, T (&part)[NR]) {
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
        const int k = qq * 16 + kk;
        const T a = M[r][k];
#pragma unroll
        for (int c = 0; c < NR; ++c) part[c] = fma(a, V[k][c], part[c]);
    }
}
// sum of the 4 quarter threads of a row
template <typename T, int NR>
__device__ __forceinline__ void quad_sum(T (&part)[NR]) {
#pragma unroll
    for (int c = 0; c < NR; ++c) {
        part[c] += __shfl_xor_sync(0xffffffffu, part[c], 1);
        part[c] += __shfl_xor_sync(0xffffffffu, part[c], 2);
    }
}

// part[c] = sum over this thread's quarter of k of M[r][k] V[k][c], summed over
// the 4 threads of row r (thread = 4 r + quarter)
template <typename T, int NR>
__device__ __forceinline__ void tile_gemv(const T (*M)[TB + 1], const T (*V)[NR], int r, int qq, T (&part)[NR]) {
#pragma unroll
    for (int c = 0; c < NR; ++c) part[c] = T(0);
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
        const int k = qq * 16 + kk;
        const T a = M[r][k];
#pragma unroll
        for (int c = 0; c < NR; ++c) part[c] = fma(a, V[k][c], part[c]);
    }
#pragma unroll
    for (int c = 0; c < NR; ++c) {
        part[c] += __shfl_xor_sync(0xffffffffu, part[c], 1);
        part[c] += __shfl_xor_sync(0xffffffffu, part[c], 2);
    }
}

// Triangular-solve launches that found their skip flag set (see
// gemv_skipped_count): the launch profile counts the work of the others only.
__device__ unsigned int g_trsv_skipped;

// mode 0: L (unit lower, forward)    mode 1: U (upper, backward)
// mode 2: U^T (lower, forward)       mode 3: L^T (unit upper, backward)
// Tile (i, j) of op(T): element (r, k) = op(T)[i TB + r][j TB + k].
template <typename TS, typename T>
__device__ __forceinline__ T tile_elem(const TS *C, int64_t ldc, int n, int mode, int i, int j, int r, int k) {
    const int64_t row = (int64_t)i * TB + r, col = (int64_t)j * TB + k;
    if (row >= n || col >= n) return T(0);
    return (mode <= 1) ? (T)__ldg(C + row * ldc + col) : (T)__ldg(C + col * ldc + row);
}

// DD: the walker reads the factors and the diagonal inverses as
// double-float pairs (Cd, ldcd, Dinvd) and works on the FP32 pipe; the
// update items still read C.
template <typename TS, typename T, int NR, bool DD>
__global__ void __launch_bounds__(kTrsvThreads) k_trsv(const TS *C, int64_t ldc, int n, const TS *Dinv, T *Y,
                                                        int64_t ldy, int nr, int mode, const int *skip, int *sync,
                                                        const dfloat *Cd, int64_t ldcd, const dfloat *Dinvd) {
    if (skip && *skip) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&g_trsv_skipped, 1u);
        return;
    }
    extern __shared__ __align__(16) unsigned char smraw[];
    TrsvSmem<T, NR> &sm = *reinterpret_cast<TrsvSmem<T, NR> *>(smraw);
    TrsvSmemDD<NR> &sd = *reinterpret_cast<TrsvSmemDD<NR> *>(smraw);
    __shared__ int s_ticket;
    const int tid = threadIdx.x;
    const int nblk = (n + TB - 1) / TB;
    // mode bit 2: factors of block GE (identity diagonal blocks in L, whole
    // pivot blocks on U's diagonal); bits 0-1: the pass, as above
    const bool bge = (mode & 4) != 0;
    mode &= 3;
    const bool forward = (mode == 0 || mode == 2);
    const bool unit = (mode == 0 || mode == 3);
    int *ticket = sync, *cnt = sync + 2, *ready = sync + 2 + nblk;
    const int r = tid >> 2, qq = tid & 3;   // tile_gemv roles
    // per-thread share of a tile load: 16 elements; non-transposed modes walk
    // rows (k fastest), transposed modes walk columns (r fastest)
    auto load_tile = [&](int i, int j, T (&v)[16]) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int idx = tid + e * kTrsvThreads;
            const int a = idx >> 6, b = idx & 63;
            v[e] = (mode <= 1) ? tile_elem<TS, T>(C, ldc, n, mode, i, j, a, b)
                               : tile_elem<TS, T>(C, ldc, n, mode, i, j, b, a);
        }
    };
    auto store_tile = [&](T (*M)[TB + 1], const T (&v)[16]) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int idx = tid + e * kTrsvThreads;
            const int a = idx >> 6, b = idx & 63;
            if (mode <= 1) M[a][b] = v[e];
            else M[b][a] = v[e];
        }
    };
    // the diagonal tile's triangle, unit diagonal where op(T) has one
    auto store_diag = [&](const T (&v)[16]) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int idx = tid + e * kTrsvThreads;
            const int a = idx >> 6, b = idx & 63;
            const int rr = mode <= 1 ? a : b, kk = mode <= 1 ? b : a;
            T val = v[e];
            if (bge) {
                if (unit) val = rr == kk ? T(1) : T(0);   // L_B: identity diagonal blocks; U_B: the pivot block
            } else if (rr == kk) {
                val = unit ? T(1) : val;
            } else if (forward ? kk > rr : kk < rr) {
                val = T(0);
            }
            sm.D[rr][kk] = val;
        }
    };
    // op(T_jj)^{-1} from the inverted diagonal blocks (Dinv: [L, U][block][64][64])
    auto load_inv = [&](int j, T (&v)[16]) {
        const TS *X = Dinv + ((int64_t)(unit ? 0 : 1) * nblk + j) * TB * TB;
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = (T)__ldg(X + tid + e * kTrsvThreads);
    };
    auto block_of = [&](int p) { return forward ? p : nblk - 1 - p; };
    // double-float walker: tiles of op(T) from the double-float factors, the
    // inverse of the diagonal tile from its double-float copy
    auto load_tile_d = [&](int i, int j, dfloat (&v)[16]) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int idx = tid + e * kTrsvThreads;
            const int a = idx >> 6, b = idx & 63;
            const int rr = mode <= 1 ? a : b, kk = mode <= 1 ? b : a;   // element (rr, kk) of op(T)'s tile
            const int64_t row = (int64_t)i * TB + rr, col = (int64_t)j * TB + kk;
            dfloat z(0.0f);
            if (row < n && col < n) z = (mode <= 1) ? Cd[row * ldcd + col] : Cd[col * ldcd + row];
            v[e] = z;
        }
    };
    auto load_inv_d = [&](int j, dfloat (&v)[16]) {
        const dfloat *X = Dinvd + ((int64_t)(unit ? 0 : 1) * nblk + j) * TB * TB;
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = X[tid + e * kTrsvThreads];
    };
    // element e of this thread's share is (rr, kk) of op(T)'s tile
    // (load_tile_d), or (a, b) of the row-major inverse of T_jj (load_inv_d),
    // whose transpose is the inverse of op(T)_jj in the transposed modes:
    // both land at [rr][kk]; kind 1 keeps the diagonal tile's triangle
    auto store_d = [&](float (*Mh)[kDdLd], float (*Ml)[kDdLd], const dfloat (&v)[16], int kind) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int idx = tid + e * kTrsvThreads;
            const int a = idx >> 6, b = idx & 63;
            const int rr = mode <= 1 ? a : b, kk = mode <= 1 ? b : a;
            dfloat val = v[e];
            if (kind == 1 && bge) {   // block GE: identity (L_B) or the whole pivot block (U_B)
                if (unit) val = rr == kk ? dfloat(1.0f) : dfloat(0.0f);
            } else if (kind == 1) {   // the diagonal tile: its triangle, unit diagonal where op(T) has one
                if (rr == kk) val = unit ? dfloat(1.0f) : val;
                else if (forward ? kk > rr : kk < rr) val = dfloat(0.0f);
            }
            Mh[rr][kk] = val.hi;
            Ml[rr][kk] = val.lo;
        }
    };

    int q_it = 2, t_base = 1;              // first ticket of target step q_it's items
    for (;;) {
        __syncthreads();
        if (tid == 0) s_ticket = atomicAdd(ticket, 1);
        __syncthreads();
        const int t = s_ticket;
        if (DD && t == 0) {
            // ---- the walker in double-float (FP32 pipe; FP64 is 64 times
            // slower on this GPU): the same steps as the FP64 walker below ----
            dfloat vD[16], vX[16], vO[16];
            // b_j of the coming step, in registers: its loads go out at the end
            // of the previous step, before the product for the next block, and
            // have landed by the time it is used
            constexpr int kBv = (TB * NR + kTrsvThreads - 1) / kTrsvThreads;
            double bv[kBv];
            auto load_b = [&](int jb) {
                const int bb = min(TB, n - jb * TB);
#pragma unroll
                for (int e = 0; e < kBv; ++e) {
                    const int idx = tid + e * kTrsvThreads;
                    const int rr = idx / NR, c = idx % NR;
                    bv[e] = (idx < TB * NR && rr < bb && c < nr) ? (double)ldcg(Y + ((int64_t)jb * TB + rr) * ldy + c)
                                                                  : 0.0;
                }
            };
            load_tile_d(block_of(0), block_of(0), vD);
            load_inv_d(block_of(0), vX);
            load_b(block_of(0));
            for (int q = 0; q < nblk; ++q) {
                const int j = block_of(q);
                const int bj = min(TB, n - j * TB);
                __syncthreads();
                store_d(sd.Dh, sd.Dl, vD, 1);
                store_d(sd.Sh, sd.Sl, vX, 2);
#pragma unroll
                for (int e = 0; e < kBv; ++e) {
                    const int idx = tid + e * kTrsvThreads;
                    if (idx < TB * NR) {
                        const int rr = idx / NR, c = idx % NR;
                        const dfloat b(bv[e]);
                        sd.acc[rr][c] = q > 0 ? b - sd.carry[rr][c] : b;
                    }
                }
                if (q + 1 < nblk) {
                    load_tile_d(block_of(q + 1), j, vO);
                    load_tile_d(block_of(q + 1), block_of(q + 1), vD);
                    load_inv_d(block_of(q + 1), vX);
                }
                __syncthreads();
                // y = X b;  y += X (b - T y)
                dfloat part[NR];
                tile_gemv_dd<NR>(sd.Sh, sd.Sl, sd.acc, r, qq, part);
#pragma unroll
                for (int c = 0; c < NR; ++c)
                    if ((c & 3) == qq) sd.y[r][c] = part[c];
                __syncthreads();
                tile_gemv_dd<NR>(sd.Dh, sd.Dl, sd.y, r, qq, part);
#pragma unroll
                for (int c = 0; c < NR; ++c)
                    if ((c & 3) == qq) sd.acc[r][c] = sd.acc[r][c] - part[c];
                __syncthreads();
                tile_gemv_dd<NR>(sd.Sh, sd.Sl, sd.acc, r, qq, part);
#pragma unroll
                for (int c = 0; c < NR; ++c)
                    if ((c & 3) == qq) {
                        const dfloat yv = sd.y[r][c] + part[c];
                        sd.y[r][c] = yv;
                        if (r < bj && c < nr) Y[((int64_t)j * TB + r) * ldy + c] = (T)(double)yv;
                    }
                __syncthreads();
                if (tid == 0) publish(ready + j);
                if (q + 1 < nblk) {           // own contribution to the next block
                    store_d(sd.Oh, sd.Ol, vO, 0);
                    // the next step's items (earlier steps up to q - 1), then its b
                    if (tid == 0 && q >= 1 && !wait_geq(cnt + block_of(q + 1), q)) atomicExch(&g_solve_timeout, 1);
                    __syncthreads();
                    load_b(block_of(q + 1));
                    tile_gemv_dd<NR>(sd.Oh, sd.Ol, sd.y, r, qq, part);
#pragma unroll
                    for (int c = 0; c < NR; ++c)
                        if ((c & 3) == qq) sd.carry[r][c] = part[c];
                }
            }
            continue;
        }
        if (t == 0) {
            // ---- the walker: every diagonal block in order ----
            T vD[16], vX[16], vO[16];
            load_tile(block_of(0), block_of(0), vD);
            load_inv(block_of(0), vX);
            for (int q = 0; q < nblk; ++q) {
                const int j = block_of(q);
                const int bj = min(TB, n - j * TB);
                __syncthreads();
                store_diag(vD);
                store_tile(sm.S, vX);
                // wait for the items of steps up to q - 2, then b_j = Y_j - own carry
                if (tid == 0 && q >= 2 && !wait_geq(cnt + j, q - 1)) atomicExch(&g_solve_timeout, 1);
                __syncthreads();
                // b_j first: its loads must not queue behind the next step's tiles
                for (int idx = tid; idx < TB * NR; idx += kTrsvThreads) {
                    const int rr = idx / NR, c = idx % NR;
                    const T b = (rr < bj && c < nr) ? ldcg(Y + ((int64_t)j * TB + rr) * ldy + c) : T(0);
                    sm.acc[rr][c] = q > 0 ? b - sm.carry[rr][c] : b;
                }
                if (q + 1 < nblk) {           // next step's tiles, in flight during this one
                    load_tile(block_of(q + 1), j, vO);
                    load_tile(block_of(q + 1), block_of(q + 1), vD);
                    load_inv(block_of(q + 1), vX);
                }
                __syncthreads();
                // y = X b;  y += X (b - T y)  (one refinement step of the explicit inverse)
                T part[NR];
                tile_gemv<T, NR>(sm.S, sm.acc, r, qq, part);
#pragma unroll
                for (int c = 0; c < NR; ++c)
                    if ((c & 3) == qq) sm.y[r][c] = part[c];
                __syncthreads();
                tile_gemv<T, NR>(sm.D, sm.y, r, qq, part);
#pragma unroll
                for (int c = 0; c < NR; ++c)
                    if ((c & 3) == qq) sm.acc[r][c] -= part[c];
                __syncthreads();
                tile_gemv<T, NR>(sm.S, sm.acc, r, qq, part);
#pragma unroll
                for (int c = 0; c < NR; ++c)
                    if ((c & 3) == qq) {
                        const T yv = sm.y[r][c] + part[c];
                        sm.y[r][c] = yv;
                        if (r < bj && c < nr) Y[((int64_t)j * TB + r) * ldy + c] = yv;
                    }
                __syncthreads();
                if (tid == 0) publish(ready + j);
                if (q + 1 < nblk) {           // own contribution to the next block
                    store_tile(sm.O, vO);
                    __syncthreads();
                    tile_gemv<T, NR>(sm.O, sm.y, r, qq, part);
#pragma unroll
                    for (int c = 0; c < NR; ++c)
                        if ((c & 3) == qq) sm.carry[r][c] = part[c];
                }
            }
            continue;
        }
        // ---- an update item: target step q, earlier steps p0 .. p1 ----
        while (q_it < nblk && t >= t_base + nchunks(q_it)) {
            t_base += nchunks(q_it);
            ++q_it;
        }
        if (q_it >= nblk) break;
        const int i = block_of(q_it);
        const int p0 = (t - t_base) * kSeg, p1 = min(q_it - 2, p0 + kSeg - 1);
        T v[16];
        load_tile(i, block_of(p0), v);
        T part[NR];
#pragma unroll
        for (int c = 0; c < NR; ++c) part[c] = T(0);
        for (int pp = p0; pp <= p1; ++pp) {
            const int j = block_of(pp);
            const int bj = min(TB, n - j * TB);
            if (tid == 0 && !wait_geq(ready + j, 1)) atomicExch(&g_solve_timeout, 1);
            __syncthreads();
            store_tile(sm.S, v);
            for (int idx = tid; idx < TB * NR; idx += kTrsvThreads) {
                const int rr = idx / NR, c = idx % NR;
                sm.y[rr][c] = (rr < bj && c < nr) ? ldcg(Y + ((int64_t)j * TB + rr) * ldy + c) : T(0);
            }
            __syncthreads();
            if (pp < p1) load_tile(i, block_of(pp + 1), v);
            tile_gemv_acc<T, NR>(sm.S, sm.y, r, qq, part);
        }
        quad_sum<T, NR>(part);
        const int64_t row = (int64_t)i * TB + r;
        if (row < n) {
#pragma unroll
            for (int c = 0; c < NR; ++c)
                if ((c & 3) == qq && c < nr) atomicAdd(Y + row * ldy + c, -part[c]);
        }
        __syncthreads();
        if (tid == 0) {       // release: the CTA's updates above, ordered by the barrier
            __threadfence();
            atomicAdd(cnt + i, p1 - p0 + 1);
        }
    }
}

// Inverses of the 64 x 64 diagonal blocks of L (unit lower, blockIdx.y = 0)
// and U (upper, blockIdx.y = 1), by column-wise substitution in FP64, stored
// row-major per block; rows and columns past a ragged last block are zero.
template <typename TS>
__global__ void __launch_bounds__(TB) k_trtri_diag(const TS *C, int64_t ldc, int n, TS *Dinv) {
    extern __shared__ __align__(16) unsigned char smraw[];
    double(*t)[TB + 1] = reinterpret_cast<double(*)[TB + 1]>(smraw);
    double(*x)[TB + 1] = t + TB;
    const int j = blockIdx.x, which = blockIdx.y, c = threadIdx.x;
    const int nblk = (n + TB - 1) / TB, bj = min(TB, n - j * TB);
    const int64_t j0 = (int64_t)j * TB;
    for (int r = 0; r < TB; ++r) t[r][c] = (r < bj && c < bj) ? (double)C[(j0 + r) * ldc + j0 + c] : 0.0;
    __syncthreads();
    for (int r = 0; r < TB; ++r) x[r][c] = 0.0;
    if (c < bj) {
        if (which == 0) {   // L x = e_c, unit diagonal
            x[c][c] = 1.0;
            for (int r = c + 1; r < bj; ++r) {
                double sum = 0.0;
                for (int k = c; k < r; ++k) sum = fma(t[r][k], x[k][c], sum);
                x[r][c] = -sum;
            }
        } else {            // U x = e_c
            x[c][c] = 1.0 / t[c][c];
            for (int r = c - 1; r >= 0; --r) {
                double sum = 0.0;
                for (int k = r + 1; k <= c; ++k) sum = fma(t[r][k], x[k][c], sum);
                x[r][c] = -sum / t[r][r];
            }
        }
    }
    __syncthreads();
    TS *out = Dinv + ((int64_t)which * nblk + j) * TB * TB;
    for (int r = 0; r < TB; ++r) out[r * TB + c] = (TS)x[r][c];
}

template <typename TS, typename T, int NR, bool DD>
cudaError_t launch_trsv(const TS *C, int64_t ldc, int64_t n, const TS *Dinv, T *Y, int64_t ldy, int nr, int mode,
                        const int *skip, int *sync, const dfloat *Cd, int64_t ldcd, const dfloat *Dinvd,
                        cudaStream_t s) {
    const size_t sm = (DD && sizeof(TrsvSmemDD<NR>) > sizeof(TrsvSmem<T, NR>)) ? sizeof(TrsvSmemDD<NR>)
                                                                               : sizeof(TrsvSmem<T, NR>);
    static int grid = 0;
    if (!grid) {
        if (sm > 48 * 1024)
            cudaFuncSetAttribute(k_trsv<TS, T, NR, DD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        int per_sm = 1, dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trsv<TS, T, NR, DD>, kTrsvThreads, sm) !=
                cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        grid = sms * per_sm;
    }
    const int64_t nblk = cdiv(n, TB);
    cudaError_t e = cudaMemsetAsync(sync, 0, (size_t)(2 + 2 * nblk) * sizeof(int), s);
    if (e != cudaSuccess) return e;
    // algorithmic bytes: the triangle of the factor read once (double-float
    // pairs are 8 B like FP64)
    auto *ev = profile_class_slot(kProfTrsv, 0.5 * (double)n * (double)n * (DD ? 8.0 : (double)sizeof(TS)));
    prof_begin(ev, s);
    note_launch();
    k_trsv<TS, T, NR, DD><<<grid, kTrsvThreads, sm, s>>>(C, ldc, (int)n, Dinv, Y, ldy, nr, mode, skip, sync, Cd,
                                                          ldcd, Dinvd);
    prof_end(ev, s);
    return cudaGetLastError();
}

template <typename TS, typename T>
cudaError_t solve_typed(const genp_factors *F, T *Y, int64_t ldy, int64_t nrhs, bool transposed, const int *skip,
                        cudaStream_t s) {
    const TS *C = static_cast<const TS *>(F->C);
    const int64_t n = F->n, ldc = F->ldc;
    if (n > INT32_MAX - TB) return cudaErrorInvalidValue;
    for (int64_t c0 = 0; c0 < nrhs; c0 += kTrsvMaxRhs) {
        const int nr = (int)(nrhs - c0 < kTrsvMaxRhs ? nrhs - c0 : kTrsvMaxRhs);
        T *Yc = Y + c0;
        for (int pass = 0; pass < 2; ++pass) {
            // pass 0: L (or U^T) forward; pass 1: U (or L^T) backward
            const int mode = (transposed ? (pass == 0 ? 2 : 3) : (pass == 0 ? 0 : 1)) | (F->block ? 4 : 0);
            const TS *D = static_cast<const TS *>(F->dinv);
            int *sy = F->trsv_sync;
            cudaError_t e = cudaSuccess;
            // factors also held as double-float pairs (sliced path): the walker runs in double-float
            const dfloat *Wd = static_cast<const dfloat *>(F->W);
            const dfloat *Dd = static_cast<const dfloat *>(F->dinv_df);
            bool dd = false;
            if constexpr (sizeof(TS) == 8) dd = Wd && Dd;
            if constexpr (sizeof(TS) == 8) {
                const int64_t lw = F->ldw;
                if (!dd) {
                } else if (nr == 1) {
                    e = launch_trsv<TS, T, 1, true>(C, ldc, n, D, Yc, ldy, nr, mode, skip, sy, Wd, lw, Dd, s);
                } else if (nr <= 2) {
                    e = launch_trsv<TS, T, 2, true>(C, ldc, n, D, Yc, ldy, nr, mode, skip, sy, Wd, lw, Dd, s);
                } else if (nr <= 4) {
                    e = launch_trsv<TS, T, 4, true>(C, ldc, n, D, Yc, ldy, nr, mode, skip, sy, Wd, lw, Dd, s);
                } else if (nr <= 8) {
                    e = launch_trsv<TS, T, 8, true>(C, ldc, n, D, Yc, ldy, nr, mode, skip, sy, Wd, lw, Dd, s);
                } else {
                    e = launch_trsv<TS, T, 16, true>(C, ldc, n, D, Yc, ldy, nr, mode, skip, sy, Wd, lw, Dd, s);
                }
            }
            if (!dd) {
                if (nr == 1) e = launch_trsv<TS, T, 1, false>(C, ldc, n, D, Yc, ldy, nr, mode, skip, sy, nullptr, 0,
                                                               nullptr, s);
                else if (nr <= 2) e = launch_trsv<TS, T, 2, false>(C, ldc, n, D, Yc, ldy, nr, mode, skip, sy, nullptr,
                                                                    0, nullptr, s);
                else if (nr <= 4) e = launch_trsv<TS, T, 4, false>(C, ldc, n, D, Yc, ldy, nr, mode, skip, sy, nullptr,
                                                                    0, nullptr, s);
                else if (nr <= 8) e = launch_trsv<TS, T, 8, false>(C, ldc, n, D, Yc, ldy, nr, mode, skip, sy, nullptr,
                                                                    0, nullptr, s);
                else e = launch_trsv<TS, T, 16, false>(C, ldc, n, D, Yc, ldy, nr, mode, skip, sy, nullptr, 0, nullptr,
                                                        s);
            }
            if (e != cudaSuccess) return e;
        }
    }
    return cudaGetLastError();
}

}  // namespace

unsigned int trsv_skipped_count(bool reset) {
    unsigned int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_trsv_skipped, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (reset) {
        const unsigned int z = 0;
        cudaMemcpyToSymbol(g_trsv_skipped, &z, sizeof(z));
    }
    return v;
}


template <typename T>
cudaError_t lu_solve_inplace(const genp_factors *F, T *Y, int64_t ldy, int64_t nrhs, bool transposed, const int *skip,
                             cudaStream_t s) {
    if (sizeof(T) == 8) {
        if (!f64_factors(F->prec)) return cudaErrorInvalidValue;
        return solve_typed<T, T>(F, Y, ldy, nrhs, transposed, skip, s);
    }
    if (f64_factors(F->prec)) return cudaErrorInvalidValue;
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

int solve_timeout_flag(bool reset) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_solve_timeout, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    if (reset && v) {
        int z = 0;
        cudaMemcpyToSymbol(g_solve_timeout, &z, sizeof(int));
    }
    return v;
}

int64_t trsv_sync_ints(int64_t n) { return 2 + 2 * cdiv(n, TB); }
int64_t diag_inverse_elems(int64_t n) { return 2 * cdiv(n, TB) * TB * TB; }

cudaError_t invert_diag_blocks(genp_factors *F, cudaStream_t s) {
    const int64_t n = F->n;
    if (n > INT32_MAX - TB) return cudaErrorInvalidValue;
    dim3 g((unsigned)cdiv(n, TB), 2);
    const size_t sm = 2 * TB * (TB + 1) * sizeof(double);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_trtri_diag<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaFuncSetAttribute(k_trtri_diag<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        attr = true;
    }
    note_launch();
    if (f64_factors(F->prec))
        k_trtri_diag<double><<<g, TB, sm, s>>>(static_cast<const double *>(F->C), F->ldc, (int)n,
                                               static_cast<double *>(F->dinv));
    else
        k_trtri_diag<float><<<g, TB, sm, s>>>(static_cast<const float *>(F->C), F->ldc, (int)n,
                                              static_cast<float *>(F->dinv));
    if (F->dinv_df) {   // double-float copy for the walker of the sliced path
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return df_from_f64(static_cast<const double *>(F->dinv), TB, static_cast<dfloat *>(F->dinv_df), TB,
                           2 * cdiv(n, TB) * TB, TB, s);
    }
    return cudaGetLastError();
}

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
    auto *ev = profile_class_slot(kProfOuter, (double)n * (double)n * (dA_f32 ? 4.0 : 8.0));
    prof_begin(ev, s);
    if (nrhs <= 4 && cdiv(n, 32) <= 65535) {
        const dim3 gr((unsigned)cdiv(n, 1024), (unsigned)cdiv(n, 32));
        const int vec = (ldda % 4 == 0) && ((uintptr_t)dA % 32 == 0);
        note_launch();
        if (dA_f32) {
            if (nrhs == 1) k_outer_rows<float, 1><<<gr, 256, 0, s>>>(Lam, ldl, X, ldx, n, 1, (float *)dA, ldda, vec);
            else k_outer_rows<float, 4><<<gr, 256, 0, s>>>(Lam, ldl, X, ldx, n, (int)nrhs, (float *)dA, ldda, vec);
        } else {
            if (nrhs == 1) k_outer_rows<double, 1><<<gr, 256, 0, s>>>(Lam, ldl, X, ldx, n, 1, (double *)dA, ldda, vec);
            else k_outer_rows<double, 4><<<gr, 256, 0, s>>>(Lam, ldl, X, ldx, n, (int)nrhs, (double *)dA, ldda, vec);
        }
    } else if (dA_f32) {
        note_launch();
        k_outer<float><<<g, 256, 0, s>>>(Lam, ldl, X, ldx, n, (int)nrhs, (float *)dA, ldda);
    } else {
        note_launch();
        k_outer<double><<<g, 256, 0, s>>>(Lam, ldl, X, ldx, n, (int)nrhs, (double *)dA, ldda);
    }
    prof_end(ev, s);
    return cudaGetLastError();
}

}  // namespace genp
