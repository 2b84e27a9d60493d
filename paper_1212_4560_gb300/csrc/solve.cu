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
// inverse of the diagonal tile plus one refinement step (the double-float
// walker: the inverse alone, see kDdBlockRefine), publishes y_j (into a
// buffer filled with an all-ones NaN before the launch, which no result
// takes: a reader sees each value land without a fence or flag), and
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
// on.  In double-float (the sliced path's factors) the walker's tiles (the
// inverse, the masked diagonal block when it refines, the next block's tile)
// come by TMA a step before they are needed, into shared memory: one SM's
// own loads of three 32 KiB tiles per step were what set the pace.
// ---------------------------------------------------------------------------
constexpr int TB = 64;          // tile
// The double-float walker's diagonal blocks: y = T_jj^{-1} b by the inverse
// alone, or followed by one refinement step y += T_jj^{-1} (b - T_jj y).
// The inverses are FP64's held to 48 bits, so the inverse alone leaves a
// block's solve within about cond(T_jj) 2^-48 (relative), the size of the
// sliced factors' own error, which the FP64 refinement that follows every
// sliced solve absorbs; the step doubled the chain's work per block.
constexpr bool kDdBlockRefine = false;
constexpr int kSeg = 16;        // tiles per work item
constexpr int kTrsvThreads = 256;
constexpr long long kSpinTicks = 4000000000LL;   // ~2 s at 2 GHz

__device__ int g_solve_timeout;

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// The published y values: relaxed (GPU scope, single-copy atomic) stores and
// loads of the value itself; the empty mark is all-ones, which a published
// value never is (a NaN with that bit pattern goes out as the default NaN).
__device__ __forceinline__ void publish_y(double *p, double v) {
    long long b = __double_as_longlong(v);
    if (b == -1LL) b = 0x7ff8000000000000LL;
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(b) : "memory");
}
__device__ __forceinline__ void publish_y(float *p, float v) {
    unsigned b = __float_as_uint(v);
    if (b == 0xffffffffu) b = 0x7fc00000u;
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(b) : "memory");
}
__device__ __forceinline__ bool load_y(const double *p, double &v) {
    long long b;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(b) : "l"(p) : "memory");
    v = __longlong_as_double(b);
    return b != -1LL;
}
__device__ __forceinline__ bool load_y(const float *p, float &v) {
    unsigned b;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(b) : "l"(p) : "memory");
    v = __uint_as_float(b);
    return b != 0xffffffffu;
}
// double-float values go out as one 8-byte word (hi, lo)
__device__ __forceinline__ void publish_y(dfloat *p, dfloat v) {
    unsigned long long b = ((unsigned long long)__float_as_uint(v.lo) << 32) | __float_as_uint(v.hi);
    if (b == ~0ull) b = 0x7fc00000ull;
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(b) : "memory");
}
__device__ __forceinline__ bool load_y(const dfloat *p, dfloat &v) {
    unsigned long long b;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(b) : "l"(p) : "memory");
    v.hi = __uint_as_float((unsigned)b);
    v.lo = __uint_as_float((unsigned)(b >> 32));
    return b != ~0ull;
}
// a published value, waiting (bounded) for it to land
template <typename T>
__device__ T wait_y(const T *p) {
    T v;
    if (load_y(p, v)) return v;
    const long long t0 = clock64();
    while (!load_y(p, v)) {
        if (clock64() - t0 > kSpinTicks) {
            atomicExch(&g_solve_timeout, 1);
            return T(0);
        }
        __nanosleep(32);
    }
    return v;
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

// Row stride of the shared right-hand-side blocks [64][NR]: a warp's tile
// products read four rows k at once, which share a bank when NR is a
// multiple of 8; one pad element keeps them apart.
template <int NR>
constexpr int kNrp = NR % 8 == 0 ? NR + 1 : NR;
// Unrolling of the tile products' k loops: whole for a few right-hand
// sides; for 8 or more the 16 x NR fully unrolled bodies at every call site
// no longer fit the instruction cache and ran four times slower.
template <int NR>
constexpr int kUnrollK = NR >= 8 ? 2 : 16;
// The double-float path's update items sum in double-float from 8
// right-hand sides on, in FP64 below.
template <int NR>
constexpr bool kDdItems = NR >= 8;

// The published block j of y (bj rows, nr of NR columns) into the shared
// [64][kNrp] block V, zero elsewhere: every thread's loads go out together,
// and only values not there yet are waited for.
template <int NR, typename T>
__device__ __forceinline__ void gather_y(T (*V)[kNrp<NR>], const T *yp, int j, int bj, int nr, int tid) {
    constexpr int kYv = (TB * NR + kTrsvThreads - 1) / kTrsvThreads;
    T v[kYv];
    bool got[kYv];
#pragma unroll
    for (int e = 0; e < kYv; ++e) {
        const int idx = tid + e * kTrsvThreads, rr = idx / NR, c = idx % NR;
        v[e] = T(0.0f);
        got[e] = true;
        if (idx < TB * NR && rr < bj && c < nr) got[e] = load_y(yp + ((int64_t)j * TB + rr) * NR + c, v[e]);
    }
#pragma unroll
    for (int e = 0; e < kYv; ++e) {
        const int idx = tid + e * kTrsvThreads, rr = idx / NR, c = idx % NR;
        if (!got[e]) v[e] = wait_y(yp + ((int64_t)j * TB + rr) * NR + c);
        if (idx < TB * NR) V[rr][c] = v[e];
    }
}

template <typename T, int NR>
struct TrsvSmem {
    T S[TB][TB + 1];    // op(T_jj)^{-1} (walker) or the current tile (items)
    T D[TB][TB + 1];    // op(T_jj), its triangle only (walker)
    T O[TB][TB + 1];    // op(T)[next][j] (walker)
    T y[TB][kNrp<NR>];        // y_j
    T acc[TB][kNrp<NR>];      // right-hand side of the diagonal block, then its residual
    T carry[TB][kNrp<NR>];    // the walker's own contribution to the next block
};

// The walker's shared memory when it runs in double-float (factors held as
// double-float pairs, GENP_BF16_SLICED).  Its tiles are kept as they lie in
// memory (rows of C, or of the row-major inverse of T_jj), so that each
// 64-pair row arrives by one bulk copy (TMA) issued a step ahead; the
// transposed modes read them transposed.  A row stride of 68 pairs keeps the
// tile products' reads free of bank conflicts either way (with the quarters
// interleaved along k, k = quarter + 4 kk, a half warp's 4 rows x 4 quarters
// hit 16 different 8-byte bank pairs).  X is double-buffered by step parity:
// step q + 2's inverse goes out as soon as step q has used its own.
constexpr int kDdLd = 68;
template <int NR>
struct TrsvSmemDD {
    alignas(128) dfloat X[2][TB][kDdLd];   // T_jj^{-1}
    alignas(128) dfloat D[TB][kDdLd];      // T_jj, its triangle with op(T)'s diagonal
    alignas(128) dfloat O[TB][kDdLd];      // the tile of op(T)[next][j], as it lies in C
    dfloat y[TB][kNrp<NR>], acc[TB][kNrp<NR>], carry[TB][kNrp<NR>];
    unsigned long long bar[4];             // tile arrivals: X[0], X[1], D, O
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void bar_init(unsigned long long *b) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void bar_expect(unsigned long long *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bar_arrive(unsigned long long *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool bar_test(unsigned long long *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded: false after ~2 s
__device__ bool bar_wait(unsigned long long *b, uint32_t parity) {
    const long long t0 = clock64();
    while (!bar_test(b, parity))
        if (clock64() - t0 > kSpinTicks) return false;
    return true;
}
// a 64 x 68 box of 8-byte elements at column x, row y of the map's matrix,
// global -> shared by TMA (rows of 68 elements land one after the other,
// which gives the tile its padded row stride; elements past the matrix read
// as zero), completing on b
constexpr uint32_t kDdTileBytes = TB * kDdLd * 8;
__device__ __forceinline__ void tma_tile(void *dst, const CUtensorMap *map, int x, int y, unsigned long long *b) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(b))
        : "memory");
}

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

// part[c] = sum_k M(r, k) V[k][c] in double-float, summed over the 4 quarter
// threads of row r (thread = 4 r + quarter), for a tile held as pairs:
// M(r, k) = M[r][k], or M[k][r] when TR.
template <int NR, bool TR>
__device__ __forceinline__ void tile_gemv_dd(const dfloat (*M)[kDdLd], const dfloat (*V)[kNrp<NR>], int r, int qq,
                                             dfloat (&part)[NR]) {
    float s[NR], t[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) s[c] = t[c] = 0.f;
#pragma unroll kUnrollK<NR>
    for (int kk = 0; kk < 16; ++kk) {
        const int k = qq + 4 * kk;
        const dfloat a = TR ? M[k][r] : M[r][k];
#pragma unroll
        for (int c = 0; c < NR; ++c) dd_mac(s[c], t[c], a.hi, a.lo, V[k][c]);
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
__device__ __forceinline__ void tile_gemv_acc(const T (*M)[TB + 1], const T (*V)[kNrp<NR>], int r, int qq,
                                              T (&part)[NR]) {
#pragma unroll kUnrollK<NR>
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
__device__ __forceinline__ void tile_gemv(const T (*M)[TB + 1], const T (*V)[kNrp<NR>], int r, int qq, T (&part)[NR]) {
#pragma unroll
    for (int c = 0; c < NR; ++c) part[c] = T(0);
#pragma unroll kUnrollK<NR>
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
__global__ void __launch_bounds__(kTrsvThreads, 1) k_trsv(const TS *C, int64_t ldc, int n, const TS *Dinv, T *Y,
                                                        int64_t ldy, int nr, int mode, const int *skip, int *sync,
                                                        T *ypub, const dfloat *Cd, int64_t ldcd, const dfloat *Dinvd,
                                                        const __grid_constant__ CUtensorMap tmC,
                                                        const __grid_constant__ CUtensorMap tmX) {
    if (skip && *skip) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&g_trsv_skipped, 1u);
        return;
    }
    extern __shared__ __align__(16) unsigned char smraw[];
    TrsvSmem<T, NR> &sm = *reinterpret_cast<TrsvSmem<T, NR> *>(smraw);
    // the walker's tiles are TMA destinations: 128-byte aligned
    TrsvSmemDD<NR> &sd = *reinterpret_cast<TrsvSmemDD<NR> *>(((uintptr_t)smraw + 127) & ~(uintptr_t)127);
    __shared__ int s_ticket;
    const int tid = threadIdx.x;
    const int nblk = (n + TB - 1) / TB;
    // mode bit 2: factors of block GE (identity diagonal blocks in L, whole
    // pivot blocks on U's diagonal); bits 0-1: the pass, as above
    const bool bge = (mode & 4) != 0;
    // bit 3: tmC and tmX map the double-float factors and the inverses, so
    // the walker's tiles come by TMA
    const bool tma = (mode & 8) != 0;
    mode &= 3;
    const bool forward = (mode == 0 || mode == 2);
    const bool unit = (mode == 0 || mode == 3);
    int *ticket = sync, *cnt = sync + 2;
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
    // double-float walker: the 64 x 64 tile at row r0, column c0 of the
    // row-major pair matrix P (leading dimension ldp, prow x pcol) into M as
    // it lies there, by one TMA box from map (thread 32) completing on bar,
    // or, without maps, by plain loads with zero fill past the matrix and one
    // arrival on bar.  Called by all threads alike.
    auto issue_tile = [&](dfloat (*M)[kDdLd], const CUtensorMap *map, const dfloat *P, int64_t ldp, int64_t prow,
                          int64_t pcol, int64_t r0, int64_t c0, unsigned long long *bar) {
        if (tma) {
            if (tid == 32) {
                // the tile's last readers are ordered before this by a block barrier
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                bar_expect(bar, kDdTileBytes);
                tma_tile(&M[0][0], map, (int)c0, (int)r0, bar);
            }
        } else {
            for (int idx = tid; idx < TB * TB; idx += kTrsvThreads) {
                const int rr = idx >> 6, cc = idx & 63;
                M[rr][cc] = (r0 + rr < prow && c0 + cc < pcol) ? P[(r0 + rr) * ldp + c0 + cc] : dfloat(0.0f);
            }
            if (tid == 0) bar_arrive(bar);
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
            // slower on this GPU): the same steps as the FP64 walker below,
            // its tiles in shared memory a step before they are needed (one
            // SM's own loads could not bring three 32 KiB tiles per step in
            // time) ----
            const bool tr = mode >= 2;
            if (tid == 0) {
                for (int b = 0; b < 4; ++b) bar_init(&sd.bar[b]);
                asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            }
            __syncthreads();
            // phases: the k-th fill of a buffer completes phase k of its barrier;
            // bit b of wpar is the parity of buffer b's next wait, of ipar that
            // of its next fill, of filled whether it has had one
            uint32_t wpar = 0, ipar = 0, filled = 0;
            bool late = false;
            auto take = [&](int b) {     // wait for the next fill of buffer b
                if (!bar_wait(&sd.bar[b], (wpar >> b) & 1u)) {
                    late = true;
                    if (tid == 0) atomicExch(&g_solve_timeout, 1);
                }
                wpar ^= 1u << b;
            };
            auto filled_one = [&](int b) {
                ipar ^= 1u << b;
                filled |= 1u << b;
            };
            // the inverses and the masked diagonal blocks, [L, U][block][64][64]
            // each, as one matrix of 64 columns
            const int64_t xrows = 4 * (int64_t)nblk * TB, xrow0 = (int64_t)(unit ? 0 : 1) * nblk * TB,
                          drow0 = xrow0 + 2 * (int64_t)nblk * TB;
            auto fill_x = [&](int q) {   // T_jj^{-1} of step q into X[q & 1]
                issue_tile(sd.X[q & 1], &tmX, Dinvd, TB, xrows, TB, xrow0 + (int64_t)block_of(q) * TB, 0,
                           &sd.bar[q & 1]);
                filled_one(q & 1);
            };
            auto fill_c = [&](dfloat (*M)[kDdLd], int bi, int bj, int b) {   // tile (bi, bj) of C
                issue_tile(M, &tmC, Cd, ldcd, n, n, (int64_t)bi * TB, (int64_t)bj * TB, &sd.bar[b]);
                filled_one(b);
            };
            auto fill_d = [&](int q) {
                issue_tile(sd.D, &tmX, Dinvd, TB, xrows, TB, drow0 + (int64_t)block_of(q) * TB, 0, &sd.bar[2]);
                filled_one(2);
            };
            auto fill_o = [&](int q) {   // op(T)[block of q + 1][block of q]
                const int i = block_of(q + 1), j = block_of(q);
                fill_c(sd.O, tr ? j : i, tr ? i : j, 3);
            };
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
            fill_x(0);
            if (nblk > 1) fill_x(1);
            if constexpr (kDdBlockRefine) fill_d(0);
            if (nblk > 1) fill_o(0);
            load_b(block_of(0));
            for (int q = 0; q < nblk; ++q) {
                const int j = block_of(q);
                const int bj = min(TB, n - j * TB);
#pragma unroll
                for (int e = 0; e < kBv; ++e) {
                    const int idx = tid + e * kTrsvThreads;
                    if (idx < TB * NR) {
                        const int rr = idx / NR, c = idx % NR;
                        const dfloat b(bv[e]);
                        sd.acc[rr][c] = q > 0 ? b - sd.carry[rr][c] : b;
                    }
                }
                const dfloat(*X)[kDdLd] = sd.X[q & 1];
                take(q & 1);
                __syncthreads();
                // y = X b  (then, with kDdBlockRefine, y += X (b - T y))
                dfloat part[NR];
                if (tr) tile_gemv_dd<NR, true>(X, sd.acc, r, qq, part);
                else tile_gemv_dd<NR, false>(X, sd.acc, r, qq, part);
                if constexpr (kDdBlockRefine) {
#pragma unroll
                    for (int c = 0; c < NR; ++c)
                        if ((c & 3) == qq) sd.y[r][c] = part[c];
                    take(2);
                    __syncthreads();
                    if (tr) tile_gemv_dd<NR, true>(sd.D, sd.y, r, qq, part);
                    else tile_gemv_dd<NR, false>(sd.D, sd.y, r, qq, part);
#pragma unroll
                    for (int c = 0; c < NR; ++c)
                        if ((c & 3) == qq) sd.acc[r][c] = sd.acc[r][c] - part[c];
                    __syncthreads();
                    if (q + 1 < nblk) fill_d(q + 1);      // D is free
                    if (tr) tile_gemv_dd<NR, true>(X, sd.acc, r, qq, part);
                    else tile_gemv_dd<NR, false>(X, sd.acc, r, qq, part);
                }
#pragma unroll
                for (int c = 0; c < NR; ++c)
                    if ((c & 3) == qq) {
                        const dfloat yv = kDdBlockRefine ? sd.y[r][c] + part[c] : part[c];
                        sd.y[r][c] = yv;
                        if (r < bj && c < nr) {
                            Y[((int64_t)j * TB + r) * ldy + c] = (T)(double)yv;
                            if constexpr (kDdItems<NR>)
                                publish_y(reinterpret_cast<dfloat *>(ypub) + ((int64_t)j * TB + r) * NR + c, yv);
                            else
                                publish_y(ypub + ((int64_t)j * TB + r) * NR + c, (T)(double)yv);
                        }
                    }
                __syncthreads();
                if (q + 2 < nblk) fill_x(q + 2);      // this step's X is free
                if (q + 1 < nblk) {                   // own contribution to the next block
                    take(3);
                    // the next step's items (earlier steps up to q - 1), then its b
                    if (tid == 0 && q >= 1 && !wait_geq(cnt + block_of(q + 1), q)) atomicExch(&g_solve_timeout, 1);
                    __syncthreads();
                    load_b(block_of(q + 1));
                    if (tr) tile_gemv_dd<NR, true>(sd.O, sd.y, r, qq, part);
                    else tile_gemv_dd<NR, false>(sd.O, sd.y, r, qq, part);
#pragma unroll
                    for (int c = 0; c < NR; ++c)
                        if ((c & 3) == qq) sd.carry[r][c] = part[c];
                    __syncthreads();
                    if (q + 2 < nblk) fill_o(q + 1);  // O is free
                }
            }
            // after a timed-out wait, the copies still in flight land before the
            // CTA's shared memory goes away (a later phase implies the earlier ones)
            if (late)
                for (int b = 0; b < 4; ++b)
                    if ((filled >> b) & 1u) bar_wait(&sd.bar[b], ((ipar >> b) & 1u) ^ 1u);
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
                        if (r < bj && c < nr) {
                            Y[((int64_t)j * TB + r) * ldy + c] = yv;
                            publish_y(ypub + ((int64_t)j * TB + r) * NR + c, yv);
                        }
                    }
                __syncthreads();
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
        if constexpr (DD && kDdItems<NR>) {
            // in double-float too, from the pair factors and the published
            // pairs: FP64 runs at 1/64 of the FP32 rate here, which 8 or more
            // right-hand sides feel (for fewer, the items' FP64 sums keep the
            // solve, as a preconditioner, a little more accurate: 8-9 Krylov
            // steps on the n = 16384 system against 12-13 in double-float)
            const dfloat *yp = reinterpret_cast<const dfloat *>(ypub);
            dfloat(*M)[kDdLd] = sd.X[0];
            auto load_pairs = [&](int bj, dfloat (&v)[16]) {   // tile (i, bj) of op(T), element (rr, kk)
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int idx = tid + e * kTrsvThreads;
                    const int a = idx >> 6, b = idx & 63;
                    const int rr = mode <= 1 ? a : b, kk = mode <= 1 ? b : a;
                    const int64_t row = (int64_t)i * TB + rr, col = (int64_t)bj * TB + kk;
                    dfloat z(0.0f);
                    if (row < n && col < n) z = (mode <= 1) ? Cd[row * ldcd + col] : Cd[col * ldcd + row];
                    v[e] = z;
                }
            };
            dfloat v[16];
            load_pairs(block_of(p0), v);
            float s_[NR], t_[NR];
#pragma unroll
            for (int c = 0; c < NR; ++c) s_[c] = t_[c] = 0.f;
            for (int pp = p0; pp <= p1; ++pp) {
                const int j = block_of(pp);
                const int bj = min(TB, n - j * TB);
                __syncthreads();
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int idx = tid + e * kTrsvThreads;
                    const int a = idx >> 6, b = idx & 63;
                    M[mode <= 1 ? a : b][mode <= 1 ? b : a] = v[e];
                }
                gather_y<NR>(sd.y, yp, j, bj, nr, tid);
                __syncthreads();
                if (pp < p1) load_pairs(block_of(pp + 1), v);
#pragma unroll kUnrollK<NR>
                for (int kk = 0; kk < 16; ++kk) {
                    const int k = qq + 4 * kk;
                    const dfloat a = M[r][k];
#pragma unroll
                    for (int c = 0; c < NR; ++c) dd_mac(s_[c], t_[c], a.hi, a.lo, sd.y[k][c]);
                }
            }
            const int64_t row = (int64_t)i * TB + r;
#pragma unroll
            for (int c = 0; c < NR; ++c) {
                dfloat a = df_norm(s_[c], t_[c]);
                for (int o = 1; o <= 2; o <<= 1) {
                    dfloat b;
                    b.hi = __shfl_xor_sync(0xffffffffu, a.hi, o);
                    b.lo = __shfl_xor_sync(0xffffffffu, a.lo, o);
                    a = a + b;
                }
                if ((c & 3) == qq && c < nr && row < n) atomicAdd(Y + row * ldy + c, -(T)(double)a);
            }
            __syncthreads();
            if (tid == 0) {       // release: the CTA's updates above, ordered by the barrier
                __threadfence();
                atomicAdd(cnt + i, p1 - p0 + 1);
            }
            continue;
        }
        T v[16];
        load_tile(i, block_of(p0), v);
        T part[NR];
#pragma unroll
        for (int c = 0; c < NR; ++c) part[c] = T(0);
        for (int pp = p0; pp <= p1; ++pp) {
            const int j = block_of(pp);
            const int bj = min(TB, n - j * TB);
            __syncthreads();
            store_tile(sm.S, v);
            gather_y<NR>(sm.y, ypub, j, bj, nr, tid);
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

// The double-float walker's diagonal tiles as the solves use them, after
// the inverses in its store: [L, U][block][64][64] row-major pairs, L_jj with
// its unit diagonal and U_jj's upper triangle (for block GE the identity and
// the whole pivot block), zero past n.
__global__ void k_diag_tiles_df(const dfloat *W, int64_t ldw, int n, int bge, dfloat *out) {
    const int j = blockIdx.x, which = blockIdx.y, nblk = gridDim.x;
    dfloat *o = out + ((int64_t)which * nblk + j) * TB * TB;
    for (int idx = threadIdx.x; idx < TB * TB; idx += blockDim.x) {
        const int r = idx >> 6, c = idx & 63;
        const int64_t row = (int64_t)j * TB + r, col = (int64_t)j * TB + c;
        dfloat v(0.0f);
        if (row < n && col < n) {
            const dfloat w = W[row * ldw + col];
            if (which == 0) v = (bge || r <= c) ? dfloat(r == c ? 1.0f : 0.0f) : w;
            else v = (bge || r <= c) ? w : dfloat(0.0f);
        }
        o[idx] = v;
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
    // each row's sum in four interleaved partial sums (the FP64 units' latency
    // made the single dependent chain the launch's cost); U's diagonal by its
    // reciprocals, formed once
    __shared__ double rdiag[TB];
    if (which == 1) rdiag[c] = c < bj ? 1.0 / t[c][c] : 0.0;
    __syncthreads();
    if (c < bj) {
        if (which == 0) {   // L x = e_c, unit diagonal
            x[c][c] = 1.0;
            for (int r = c + 1; r < bj; ++r) {
                double s4[4] = {0.0, 0.0, 0.0, 0.0};
                int k = c;
                for (; k + 3 < r; k += 4)
#pragma unroll
                    for (int q = 0; q < 4; ++q) s4[q] = fma(t[r][k + q], x[k + q][c], s4[q]);
                for (; k < r; ++k) s4[0] = fma(t[r][k], x[k][c], s4[0]);
                x[r][c] = -((s4[0] + s4[1]) + (s4[2] + s4[3]));
            }
        } else {            // U x = e_c
            x[c][c] = rdiag[c];
            for (int r = c - 1; r >= 0; --r) {
                double s4[4] = {0.0, 0.0, 0.0, 0.0};
                int k = r + 1;
                for (; k + 3 <= c; k += 4)
#pragma unroll
                    for (int q = 0; q < 4; ++q) s4[q] = fma(t[r][k + q], x[k + q][c], s4[q]);
                for (; k <= c; ++k) s4[0] = fma(t[r][k], x[k][c], s4[0]);
                x[r][c] = -((s4[0] + s4[1]) + (s4[2] + s4[3])) * rdiag[r];
            }
        }
    }
    __syncthreads();
    TS *out = Dinv + ((int64_t)which * nblk + j) * TB * TB;
    for (int r = 0; r < TB; ++r) out[r * TB + c] = (TS)x[r][c];
}

// The double-float walker's tensor maps: the factors' pairs (n x n) and the
// inverses' ([L, U][block][64][64] as 2 nblk 64 rows of 64), boxes of 64
// rows x 68 pairs.
struct TrsvMaps {
    CUtensorMap c, x;
    bool ok = false;
};

template <typename TS, typename T, int NR, bool DD>
cudaError_t launch_trsv(const TS *C, int64_t ldc, int64_t n, const TS *Dinv, T *Y, int64_t ldy, int nr, int mode,
                        const int *skip, int *sync, T *ypub, const dfloat *Cd, int64_t ldcd, const dfloat *Dinvd,
                        const TrsvMaps &maps, cudaStream_t s) {
    static_assert(sizeof(TrsvSmemDD<NR>) + 128 <= 227 * 1024 && sizeof(TrsvSmem<T, NR>) <= 227 * 1024,
                  "shared memory");
    // the walker aligns its part to 128 bytes
    const size_t sm = (DD && sizeof(TrsvSmemDD<NR>) + 128 > sizeof(TrsvSmem<T, NR>)) ? sizeof(TrsvSmemDD<NR>) + 128
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
    cudaError_t e = cudaMemsetAsync(sync, 0, (size_t)(2 + nblk) * sizeof(int), s);
    // the published y: all ones, the empty mark
    if (e == cudaSuccess) e = cudaMemsetAsync(ypub, 0xff, (size_t)(nblk * TB * NR) * sizeof(T), s);
    if (e != cudaSuccess) return e;
    // algorithmic bytes: the triangle of the factor read once (double-float
    // pairs are 8 B like FP64)
    auto *ev = profile_class_slot(kProfTrsv, 0.5 * (double)n * (double)n * (DD ? 8.0 : (double)sizeof(TS)));
    prof_begin(ev, s);
    note_launch();
    k_trsv<TS, T, NR, DD><<<grid, kTrsvThreads, sm, s>>>(C, ldc, (int)n, Dinv, Y, ldy, nr,
                                                          mode | (DD && maps.ok ? 8 : 0), skip, sync, ypub, Cd, ldcd,
                                                          Dinvd, maps.c, maps.x);
    prof_end(ev, s);
    return cudaGetLastError();
}

template <typename TS, typename T, bool DD>
cudaError_t launch_trsv_nr(const TS *C, int64_t ldc, int64_t n, const TS *Dinv, T *Y, int64_t ldy, int nr, int mode,
                           const int *skip, int *sync, T *yp, const dfloat *Cd, int64_t ldcd, const dfloat *Dinvd,
                           const TrsvMaps &maps, cudaStream_t s) {
    if (nr == 1)
        return launch_trsv<TS, T, 1, DD>(C, ldc, n, Dinv, Y, ldy, nr, mode, skip, sync, yp, Cd, ldcd, Dinvd, maps, s);
    if (nr <= 2)
        return launch_trsv<TS, T, 2, DD>(C, ldc, n, Dinv, Y, ldy, nr, mode, skip, sync, yp, Cd, ldcd, Dinvd, maps, s);
    if (nr <= 4)
        return launch_trsv<TS, T, 4, DD>(C, ldc, n, Dinv, Y, ldy, nr, mode, skip, sync, yp, Cd, ldcd, Dinvd, maps, s);
    if (nr <= 8)
        return launch_trsv<TS, T, 8, DD>(C, ldc, n, Dinv, Y, ldy, nr, mode, skip, sync, yp, Cd, ldcd, Dinvd, maps, s);
    return launch_trsv<TS, T, 16, DD>(C, ldc, n, Dinv, Y, ldy, nr, mode, skip, sync, yp, Cd, ldcd, Dinvd, maps, s);
}

template <typename TS, typename T>
cudaError_t solve_typed(const genp_factors *F, T *Y, int64_t ldy, int64_t nrhs, bool transposed, const int *skip,
                        cudaStream_t s) {
    const TS *C = static_cast<const TS *>(F->C);
    const int64_t n = F->n, ldc = F->ldc;
    if (n > INT32_MAX - TB) return cudaErrorInvalidValue;
    // factors also held as double-float pairs (sliced path): the walker runs in double-float
    const dfloat *Wd = static_cast<const dfloat *>(F->W);
    const dfloat *Dd = static_cast<const dfloat *>(F->dinv_df);
    const bool dd = sizeof(TS) == 8 && Wd && Dd;
    TrsvMaps maps;
    if (dd)
        maps.ok = make_map_8b(&maps.c, Wd, n, n, F->ldw, kDdLd, TB) &&
                  make_map_8b(&maps.x, Dd, 4 * cdiv(n, TB) * TB, TB, TB, kDdLd, TB);
    const TS *D = static_cast<const TS *>(F->dinv);
    int *sy = F->trsv_sync;
    T *yp = static_cast<T *>(F->trsv_y);
    for (int64_t c0 = 0; c0 < nrhs; c0 += kTrsvMaxRhs) {
        const int nr = (int)(nrhs - c0 < kTrsvMaxRhs ? nrhs - c0 : kTrsvMaxRhs);
        T *Yc = Y + c0;
        for (int pass = 0; pass < 2; ++pass) {
            // pass 0: L (or U^T) forward; pass 1: U (or L^T) backward
            const int mode = (transposed ? (pass == 0 ? 2 : 3) : (pass == 0 ? 0 : 1)) | (F->block ? 4 : 0);
            cudaError_t e;
            if constexpr (sizeof(TS) == 8) {
                if (dd) {
                    e = launch_trsv_nr<TS, T, true>(C, ldc, n, D, Yc, ldy, nr, mode, skip, sy, yp, Wd, F->ldw, Dd, maps,
                                                    s);
                    if (e != cudaSuccess) return e;
                    continue;
                }
            }
            e = launch_trsv_nr<TS, T, false>(C, ldc, n, D, Yc, ldy, nr, mode, skip, sy, yp, nullptr, 0, nullptr, maps,
                                             s);
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
    // the factors' type is the solve's: FP64 factors with FP64 vectors, FP32 with FP32
    if constexpr (sizeof(T) == 8) {
        if (!f64_factors(F->prec)) return cudaErrorInvalidValue;
        return solve_typed<T, T>(F, Y, ldy, nrhs, transposed, skip, s);
    } else {
        if (f64_factors(F->prec)) return cudaErrorInvalidValue;
        return solve_typed<float, T>(F, Y, ldy, nrhs, transposed, skip, s);
    }
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

int64_t trsv_sync_ints(int64_t n) { return 2 + cdiv(n, TB); }
int64_t trsv_y_elems(int64_t n) { return cdiv(n, TB) * TB * kTrsvMaxRhs; }
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
    if (F->dinv_df) {   // double-float copy for the walker of the sliced path, then its diagonal tiles
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        dfloat *Dd = static_cast<dfloat *>(F->dinv_df);
        e = df_from_f64(static_cast<const double *>(F->dinv), TB, Dd, TB, 2 * cdiv(n, TB) * TB, TB, s);
        if (e != cudaSuccess) return e;
        note_launch();
        k_diag_tiles_df<<<g, 256, 0, s>>>(static_cast<const dfloat *>(F->W), F->ldw, (int)n, F->block ? 1 : 0,
                                          Dd + diag_inverse_elems(n));
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
