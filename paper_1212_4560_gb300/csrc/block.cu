// block.cu -- block Gaussian elimination with explicit inverses of the pivot
// blocks (Sec. 2: Theorem 2.2 bounds the norms of the pivot blocks of block
// Gaussian elimination and of their inverses, as it bounds the pivots of
// GENP, for a strongly well conditioned matrix such as A G).
//
// C is cut into 64 x 64 diagonal blocks (the last one ragged).  Step k:
//   P_k = S_kk, the leading block of the current Schur complement, is
//         inverted explicitly by Gauss-Jordan elimination without pivoting
//         (one CTA, [P | I] in shared memory);
//   L_ik = S_ik P_k^{-1} for the block column below it (one CTA per 64 rows,
//         in place);
//   S_ij <- S_ij - L_ik S_kj for the trailing matrix (the FP64 GEMM of the
//         point factorization).
// So C = L_B U_B with L_B block unit lower (identity diagonal blocks) and U_B
// block upper with the pivot blocks on its diagonal; C holds L_B below the
// block diagonal and U_B on and above it.  The inverses go straight into the
// factors' diagonal-inverse store ([L, U][block][64][64]: identity for L_B,
// P_k^{-1} for U_B), which is what the streaming triangular solves apply at
// every diagonal block, so genp_solve, genp_refine and genp_adjoint run on
// these factors unchanged (the solve reads the diagonal tiles whole).
#include "genp_internal.cuh"

namespace genp {

namespace {

constexpr int BB = 64;               // block order = the triangular solves' tile
constexpr int kInvThreads = 1024;
constexpr int kLd = BB + 1;

struct InvSmem {
    double M[BB][kLd];               // P, reduced to I
    double X[BB][kLd];               // I, turned into P^{-1}
    double prow[2 * BB];             // row t of [M | X] divided by the pivot
    double fcol[BB];                 // column t of M before the step
};

// Gauss-Jordan on [P | I] for the kb x kb pivot block at (k0, k0).  Writes
// P^{-1} (zero-padded to 64 x 64) to Xu and the identity to Xl; folds the
// pivots into the status (a zero or non-finite pivot at step t is a
// breakdown at k0 + t; the elimination goes on, the factors are then
// meaningless, as for GENP).
__global__ void __launch_bounds__(kInvThreads) k_bge_inverse(const double *C, int64_t ldc, int64_t k0, int kb,
                                                           double *Xl, double *Xu, DevStatus *st) {
    extern __shared__ __align__(16) unsigned char smraw[];
    InvSmem &sm = *reinterpret_cast<InvSmem *>(smraw);
    const int tid = threadIdx.x;
    for (int idx = tid; idx < BB * BB; idx += kInvThreads) {
        const int r = idx / BB, c = idx % BB;
        sm.M[r][c] = (r < kb && c < kb) ? C[(k0 + r) * ldc + k0 + c] : (r == c ? 1.0 : 0.0);
        sm.X[r][c] = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    double pmin = INFINITY, pmax = 0.0;
    for (int t = 0; t < kb; ++t) {
        const double p = sm.M[t][t];
        if (tid == 0) {
            const double a = fabs(p);
            if (p == 0.0 || !isfinite(p)) atomicMin(&st->breakdown_step, (unsigned long long)(k0 + t));
            pmin = fmin(pmin, a);
            pmax = fmax(pmax, a);
        }
        if (tid < 2 * BB) sm.prow[tid] = (tid < BB ? sm.M[t][tid] : sm.X[t][tid - BB]) / p;
        else if (tid < 3 * BB) sm.fcol[tid - 2 * BB] = sm.M[tid - 2 * BB][t];
        __syncthreads();
        // 64 rows x 128 columns of [M | X], 8 entries per thread
        for (int idx = tid; idx < BB * 2 * BB; idx += kInvThreads) {
            const int r = idx / (2 * BB), c = idx % (2 * BB);
            double *e = c < BB ? &sm.M[r][c] : &sm.X[r][c - BB];
            *e = (r == t) ? sm.prow[c] : fma(-sm.fcol[r], sm.prow[c], *e);
        }
        __syncthreads();
    }
    for (int idx = tid; idx < BB * BB; idx += kInvThreads) {
        const int r = idx / BB, c = idx % BB;
        Xu[idx] = (r < kb && c < kb) ? sm.X[r][c] : 0.0;
        Xl[idx] = (r == c) ? 1.0 : 0.0;
    }
    if (tid == 0 && kb > 0) {
        atomic_min_nonneg(&st->min_abs_pivot, pmin);
        atomic_max_nonneg(&st->max_abs_pivot, pmax);
    }
}

// L_ik = S_ik P_k^{-1} in place: one CTA per 64 rows of the block column
// (rows e0 .. n-1, columns k0 .. k0+kb-1), the rows and P_k^{-1} staged in
// shared memory, 16 outputs per thread.
constexpr int kMulThreads = 256;
struct MulSmem {
    double S[BB][kLd];
    double X[BB][kLd];
};
__global__ void __launch_bounds__(kMulThreads) k_bge_lmul(double *C, int64_t ldc, int64_t n, int64_t k0, int kb,
                                                        const double *Xu) {
    extern __shared__ __align__(16) unsigned char smraw[];
    MulSmem &sm = *reinterpret_cast<MulSmem *>(smraw);
    auto &S = sm.S;
    auto &X = sm.X;
    const int64_t r0 = k0 + kb + (int64_t)blockIdx.x * BB;
    const int tid = threadIdx.x;
    for (int idx = tid; idx < BB * BB; idx += kMulThreads) {
        const int r = idx / BB, c = idx % BB;
        S[r][c] = (r0 + r < n && c < kb) ? C[(r0 + r) * ldc + k0 + c] : 0.0;
        X[r][c] = Xu[idx];
    }
    __syncthreads();
    // thread: row tr = tid / 4 (64 rows), 16 columns c = (tid % 4) + 4 q
    const int tr = tid >> 2, tc = tid & 3;
    double acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    for (int p = 0; p < kb; ++p) {
        const double s = S[tr][p];
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = fma(s, X[p][tc + 4 * q], acc[q]);
    }
    if (r0 + tr < n)
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int c = tc + 4 * q;
            if (c < kb) C[(r0 + tr) * ldc + k0 + c] = acc[q];
        }
}

// max |u_ij| over U_B (the blocks on and above the block diagonal).
__global__ void k_bge_maxu(const double *C, int64_t ldc, int64_t n, DevStatus *st) {
    double m = 0.0;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const int64_t j0 = i / BB * BB;
        for (int64_t j = j0 + threadIdx.x; j < n; j += blockDim.x) m = fmax(m, fabs(C[i * ldc + j]));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(&st->max_abs_u, m);
}

}  // namespace

cudaError_t factor_block(genp_factors *F, cudaStream_t s) {
    double *C = static_cast<double *>(F->C);
    const int64_t n = F->n, ldc = F->ldc;
    if (F->nb != BB) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_bge_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(InvSmem));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_bge_lmul, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MulSmem));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int64_t nblk = cdiv(n, BB);
    double *Xl = static_cast<double *>(F->dinv);
    double *Xu = Xl + nblk * BB * BB;
    cudaError_t em = maxabs_f64(C, n, ldc, &F->st->max_abs_c, s);
    if (em != cudaSuccess) return em;
    for (int64_t b = 0; b < nblk; ++b) {
        const int64_t k0 = b * BB;
        const int kb = (int)(n - k0 < BB ? n - k0 : BB);
        double *xu = Xu + b * BB * BB;
        auto *ev = profile_class_slot(kProfFactorAux, 2.0 * (double)kb * kb * kb);
        prof_begin(ev, s);
        note_launch();
        k_bge_inverse<<<1, kInvThreads, sizeof(InvSmem), s>>>(C, ldc, k0, kb, Xl + b * BB * BB, xu, F->st);
        prof_end(ev, s);
        const int64_t e0 = k0 + kb, rem = n - e0;
        if (rem <= 0) break;
        ev = profile_class_slot(kProfFactorAux, 2.0 * (double)rem * kb * kb);
        prof_begin(ev, s);
        note_launch();
        k_bge_lmul<<<(unsigned)cdiv(rem, BB), kMulThreads, sizeof(MulSmem), s>>>(C, ldc, n, k0, kb, xu);
        prof_end(ev, s);
        double *L21 = C + e0 * ldc + k0;
        double *U12 = C + k0 * ldc + e0;
        double *A22 = C + e0 * ldc + e0;
        cudaError_t e = gemm<double>(rem, rem, kb, -1.0, L21, ldc, false, U12, ldc, 1.0, A22, ldc, A22, ldc,
                                     nullptr, s);
        if (e != cudaSuccess) return e;
    }
    note_launch();
    k_bge_maxu<<<152 * 4, 256, 0, s>>>(C, ldc, n, F->st);
    return cudaGetLastError();
}

}  // namespace genp
