// gmres.cu -- GMRES-based iterative refinement (method 1 of genp_refine).
//
// Classic refinement (Sec. 7.1) contracts only while the factors' error,
// magnified by the element growth of pivot-free elimination, stays well below
// one.  GMRES-IR (Carson & Higham, SIAM J. Sci. Comput. 2018) keeps the same
// outer loop
//   r = b - A x (FP64);  solve C d = r;  x += G d (FP64)
// but solves the correction equation by GMRES on the left-preconditioned
// system (U^{-1} L^{-1}) C d = (U^{-1} L^{-1}) r, in FP64, with
// C v = A (G v) applied from the original A and the multiplier (C itself is
// overwritten by the factors).  With the multiplier on the left, C = G A:
// the system is C d = G r, C v = G (A v), and x += d.  The factors then need only be a good
// preconditioner, not a contraction.  Every right-hand side runs its own
// Krylov space in the same kernels (columns of the n x nrhs blocks).
//
// Arnoldi uses classical Gram-Schmidt with one reorthogonalization (CGS2);
// the Hessenberg matrix is reduced by Givens rotations as it grows, so the
// residual norm of each column's least-squares problem is known after every
// step.  All of it is steered on the device: the small kernels set a skip
// flag once every column has converged (or the outer loop has stopped), and
// the remaining enqueued kernels return at once.  Inner sums use a fixed
// reduction order (deterministic).
#include "genp_internal.cuh"

#include <math.h>

namespace genp {
namespace {

constexpr int kM = GENP_GMRES_RESTART;   // Krylov vectors per outer step
constexpr int kR = kMaxRhsChunk;         // right-hand sides per call
constexpr int kParts = 128;              // row partitions of the inner products
constexpr double kInnerTol = 1e-10;      // GMRES stops at ||res|| <= kInnerTol ||M^-1 r||

struct GmState {
    double H[kM + 1][kM][kR];
    double cs[kM][kR], sn[kM][kR], g[kM + 1][kR];
    double y[kM][kR];
    double hcol[kM + 1][kR];
    double beta[kR], scale[kR];
    int kk[kR];
    int conv[kR];
    int inner_done;
};

// partial[p][i][c] = sum over rows of partition p of V_i[r][c] * W[r][c], i < nv
__global__ void k_gm_dots(const double *V, int64_t vstride, int nv, const double *W, int64_t n, int nr,
                          double *partial, const int *skip) {
    if (*skip) return;
    __shared__ double red[8][kR];
    const int i = blockIdx.y, p = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r0 = n * p / kParts, r1 = n * (p + 1) / kParts;
    const double *Vi = V + (int64_t)i * vstride;
    double acc[kR];
#pragma unroll
    for (int c = 0; c < kR; ++c) acc[c] = 0.0;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x)
#pragma unroll
        for (int c = 0; c < kR; ++c)
            if (c < nr) acc[c] = fma(Vi[r * nr + c], W[r * nr + c], acc[c]);
#pragma unroll
    for (int c = 0; c < kR; ++c)
        for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
    if (lane == 0)
        for (int c = 0; c < kR; ++c) red[warp][c] = acc[c];
    __syncthreads();
    if (threadIdx.x < nr) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += red[w][threadIdx.x];
        partial[((int64_t)p * (kM + 1) + i) * kR + threadIdx.x] = v;
    }
    (void)nv;
}

// hcol[i][c] = sum_p partial[p][i][c]; H[i][k] (+)= hcol (add: second CGS pass)
__global__ void k_gm_reduce(GmState *st, const double *partial, int nv, int nr, int k, int add, const int *skip) {
    if (*skip) return;
    for (int idx = threadIdx.x; idx < nv * nr; idx += blockDim.x) {
        const int i = idx / nr, c = idx % nr;
        double v = 0.0;
        for (int p = 0; p < kParts; ++p) v += partial[((int64_t)p * (kM + 1) + i) * kR + c];
        st->hcol[i][c] = v;
        if (k >= 0) st->H[i][k][c] = add ? st->H[i][k][c] + v : v;
    }
}

// W[r][c] -= sum_{i < nv} V_i[r][c] hcol[i][c]
__global__ void k_gm_update(const double *V, int64_t vstride, int nv, double *W, int64_t n, int nr,
                            const GmState *st, const int *skip) {
    if (*skip) return;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * nr;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(idx % nr);
        double w = W[idx];
        for (int i = 0; i < nv; ++i) w = fma(-V[(int64_t)i * vstride + idx], st->hcol[i][c], w);
        W[idx] = w;
    }
}

// dst[r][c] = src[r][c] * scale[c]
__global__ void k_gm_scale(const double *src, double *dst, int64_t n, int nr, const GmState *st, const int *skip) {
    if (*skip) return;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * nr;
         idx += (int64_t)gridDim.x * blockDim.x)
        dst[idx] = src[idx] * st->scale[(int)(idx % nr)];
}

// New outer step: nothing converged yet; inner kernels run unless the outer loop stopped.
__global__ void k_gm_begin(GmState *st, int nr, const int *outer_done) {
    for (int c = threadIdx.x; c < kR; c += blockDim.x) {
        st->conv[c] = c < nr ? 0 : 1;
        st->kk[c] = 0;
        for (int i = 0; i <= kM; ++i) st->g[i][c] = 0.0;
    }
    if (threadIdx.x == 0) st->inner_done = *outer_done;
}

// beta_c = ||z0||, g = beta e1, scale = 1 / beta (0 for a zero residual: converged)
__global__ void k_gm_start(GmState *st, int nr, const int *skip) {
    if (*skip) return;
    const int c = threadIdx.x;
    if (c < nr) {
        const double b = sqrt(st->hcol[0][c]);
        st->beta[c] = b;
        st->g[0][c] = b;
        if (!(b > 0.0) || !isfinite(b)) {
            st->conv[c] = 1;
            st->scale[c] = 0.0;
        } else {
            st->scale[c] = 1.0 / b;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int all = 1;
        for (int q = 0; q < nr; ++q) all &= st->conv[q];
        if (all) st->inner_done = 1;
    }
}

// Arnoldi step k: h_{k+1,k} = ||w||; rotate column k of H; test convergence.
__global__ void k_gm_arnoldi(GmState *st, DevStatus *ds, int nr, int k, const int *skip) {
    if (*skip) return;
    const int c = threadIdx.x;
    if (c == 0) ds->krylov_steps += 1;
    if (c < nr && !st->conv[c]) {
        const double h = sqrt(st->hcol[0][c]);
        st->H[k + 1][k][c] = h;
        for (int i = 0; i < k; ++i) {   // earlier rotations
            const double a = st->H[i][k][c], b = st->H[i + 1][k][c];
            st->H[i][k][c] = st->cs[i][c] * a + st->sn[i][c] * b;
            st->H[i + 1][k][c] = -st->sn[i][c] * a + st->cs[i][c] * b;
        }
        const double a = st->H[k][k][c], b = st->H[k + 1][k][c];
        const double rr = hypot(a, b);
        const double cs = rr > 0.0 ? a / rr : 1.0, sn = rr > 0.0 ? b / rr : 0.0;
        st->cs[k][c] = cs;
        st->sn[k][c] = sn;
        st->H[k][k][c] = rr;
        st->H[k + 1][k][c] = 0.0;
        const double gk = st->g[k][c];
        st->g[k][c] = cs * gk;
        st->g[k + 1][c] = -sn * gk;
        const bool done = !(fabs(st->g[k + 1][c]) > kInnerTol * st->beta[c]) || !(h > 0.0) || k + 1 == kM;
        if (done) {
            st->conv[c] = 1;
            st->kk[c] = k + 1;
        }
        st->scale[c] = (done || !(h > 0.0)) ? 0.0 : 1.0 / h;
    } else if (c < nr) {
        st->scale[c] = 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int all = 1;
        for (int q = 0; q < nr; ++q) all &= st->conv[q];
        if (all) st->inner_done = 1;
    }
}

// y = H(0:kk, 0:kk)^{-1} g(0:kk) per column (back substitution)
__global__ void k_gm_finish(GmState *st, int nr, const int *outer_done) {
    if (*outer_done) return;
    const int c = threadIdx.x;
    if (c >= nr) return;
    const int kk = st->kk[c];
    for (int i = kM - 1; i >= 0; --i) {
        if (i >= kk) {
            st->y[i][c] = 0.0;
            continue;
        }
        double v = st->g[i][c];
        for (int j = i + 1; j < kk; ++j) v -= st->H[i][j][c] * st->y[j][c];
        const double d = st->H[i][i][c];
        st->y[i][c] = d != 0.0 ? v / d : 0.0;
    }
}

// D[r][c] = sum_i V_i[r][c] y[i][c]
__global__ void k_gm_combine(const double *V, int64_t vstride, double *D, int64_t n, int nr, const GmState *st,
                             const int *outer_done) {
    if (*outer_done) return;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * nr;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(idx % nr);
        double d = 0.0;
        for (int i = 0; i < st->kk[c]; ++i) d = fma(V[(int64_t)i * vstride + idx], st->y[i][c], d);
        D[idx] = d;
    }
}

unsigned vec_blocks(int64_t count) {
    const int64_t b = cdiv(count, 256);
    return (unsigned)(b < 152 * 8 ? (b < 1 ? 1 : b) : 152 * 8);
}

// w <- M^{-1} w in the factors' precision (w double, n x nr)
cudaError_t precond(const genp_factors *F, double *w, float *wf, int64_t n, int nr, const int *skip, cudaStream_t s) {
    if (f64_factors(F->prec)) return lu_solve_inplace<double>(F, w, nr, nr, false, skip, s);
    cudaError_t e = convert_matrix<double, float>(w, nr, wf, nr, n, nr, skip, s);
    if (e == cudaSuccess) e = lu_solve_inplace<float>(F, wf, nr, nr, false, skip, s);
    if (e == cudaSuccess) e = convert_matrix<float, double>(wf, nr, w, nr, n, nr, skip, s);
    return e;
}

// the inner products of W against V_0..V_{nv-1} into hcol (and H column k if k >= 0)
cudaError_t dots(GmState *st, double *partial, const double *V, int64_t vstride, int nv, const double *W, int64_t n,
                 int nr, int k, int add, const int *skip, cudaStream_t s) {
    note_launch();
    k_gm_dots<<<dim3(kParts, nv), 256, 0, s>>>(V, vstride, nv, W, n, nr, partial, skip);
    note_launch();
    k_gm_reduce<<<1, 256, 0, s>>>(st, partial, nv, nr, k, add, skip);
    return cudaGetLastError();
}

}  // namespace

size_t gmres_work_bytes(int64_t n, int64_t nrhs) {
    const size_t vec = ((size_t)n * nrhs * sizeof(double) + 255) & ~(size_t)255;
    const size_t vecf = ((size_t)n * nrhs * sizeof(float) + 255) & ~(size_t)255;
    const size_t part = ((size_t)kParts * (kM + 1) * kR * sizeof(double) + 255) & ~(size_t)255;
    const size_t stb = (sizeof(GmState) + 255) & ~(size_t)255;
    return vec * (kM + 1 + 3) + vecf + part + stb;
}

cudaError_t refine_gmres(genp_factors *F, const genp_multiplier *G, const double *A, int64_t lda, const double *B,
                         int64_t ldb, int64_t nrhs, double *X, int64_t ldx, double tol, int max_iter, void *work,
                         cudaStream_t s, CondRec *cr) {
    const int64_t n = F->n;
    const int nr = (int)nrhs;
    const size_t vec = ((size_t)n * nrhs * sizeof(double) + 255) & ~(size_t)255;
    const size_t vecf = ((size_t)n * nrhs * sizeof(float) + 255) & ~(size_t)255;
    const size_t part = ((size_t)kParts * (kM + 1) * kR * sizeof(double) + 255) & ~(size_t)255;
    char *p = static_cast<char *>(work);
    double *R = reinterpret_cast<double *>(p);
    double *V = reinterpret_cast<double *>(p + vec);              // kM + 1 vectors, vstride n * nr
    double *W = reinterpret_cast<double *>(p + vec * (kM + 2));
    double *T = reinterpret_cast<double *>(p + vec * (kM + 3));
    float *Wf = reinterpret_cast<float *>(p + vec * (kM + 4));
    double *partial = reinterpret_cast<double *>(p + vec * (kM + 4) + vecf);
    GmState *st = reinterpret_cast<GmState *>(p + vec * (kM + 4) + vecf + part);
    const int64_t vstride = n * nr;
    const int *outer_done = &F->st->refine_done;
    const int *inner = &st->inner_done;
    const unsigned vb = vec_blocks(n * nr);
    const bool left = G->side == GENP_SIDE_LEFT;
    cudaError_t e = refine_init(F, A, lda, n, s);
    for (int it = 0; it <= max_iter && e == cudaSuccess; ++it) {
        // the residual and its check, then one restarted cycle: each skipped
        // once the refinement has converged
        if (it > 0) e = cond_begin(cr, s, outer_done);
        if (e == cudaSuccess)
            e = gemm<double>(n, nrhs, n, -1.0, A, lda, false, X, ldx, 1.0, B, ldb, R, nrhs, outer_done, s);
        if (e == cudaSuccess) e = refine_check(F, R, nrhs, X, ldx, B, ldb, n, nrhs, it, tol, max_iter, 1, s);
        if (e == cudaSuccess && it > 0) e = cond_end(cr, s);
        if (e != cudaSuccess || it == max_iter) break;
        e = cond_begin(cr, s, outer_done);
        if (e != cudaSuccess) break;
        note_launch();
        k_gm_begin<<<1, 32, 0, s>>>(st, nr, outer_done);
        // V_0 = M^{-1} r / ||M^{-1} r||  (left multiplier: M^{-1} G r)
        if (left) e = apply_multiplier(G, false, R, nrhs, V, nrhs, nrhs, false, inner, s);
        else e = cudaMemcpyAsync(V, R, (size_t)n * nrhs * sizeof(double), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = precond(F, V, Wf, n, nr, inner, s);
        if (e == cudaSuccess) e = dots(st, partial, V, vstride, 1, V, n, nr, -1, 0, inner, s);
        note_launch();
        k_gm_start<<<1, 32, 0, s>>>(st, nr, inner);
        note_launch();
        k_gm_scale<<<vb, 256, 0, s>>>(V, V, n, nr, st, inner);
        for (int k = 0; k < kM && e == cudaSuccess; ++k) {
            // a Krylov step, skipped once the cycle has converged
            e = cond_begin(cr, s, inner);
            if (e != cudaSuccess) break;
            double *Vk = V + (int64_t)k * vstride;
            // W = M^{-1} A (G V_k)  (left multiplier: M^{-1} G (A V_k))
            if (left) {
                e = gemm<double>(n, nrhs, n, 1.0, A, lda, false, Vk, nrhs, 0.0, nullptr, 0, T, nrhs, inner, s);
                if (e == cudaSuccess) e = apply_multiplier(G, false, T, nrhs, W, nrhs, nrhs, false, inner, s);
            } else {
                e = apply_multiplier(G, false, Vk, nrhs, T, nrhs, nrhs, false, inner, s);
                if (e == cudaSuccess)
                    e = gemm<double>(n, nrhs, n, 1.0, A, lda, false, T, nrhs, 0.0, nullptr, 0, W, nrhs, inner, s);
            }
            if (e == cudaSuccess) e = precond(F, W, Wf, n, nr, inner, s);
            // CGS2 against V_0..V_k
            for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
                e = dots(st, partial, V, vstride, k + 1, W, n, nr, k, pass, inner, s);
                note_launch();
                k_gm_update<<<vb, 256, 0, s>>>(V, vstride, k + 1, W, n, nr, st, inner);
            }
            if (e == cudaSuccess) e = dots(st, partial, W, 0, 1, W, n, nr, -1, 0, inner, s);
            note_launch();
            k_gm_arnoldi<<<1, 32, 0, s>>>(st, F->st, nr, k, inner);
            if (k + 1 < kM) {
                note_launch();
                k_gm_scale<<<vb, 256, 0, s>>>(W, V + (int64_t)(k + 1) * vstride, n, nr, st, inner);
            }
            if (e == cudaSuccess) e = cond_end(cr, s);
        }
        if (e != cudaSuccess) break;
        // d = V y;  x += G d
        note_launch();
        k_gm_finish<<<1, 32, 0, s>>>(st, nr, outer_done);
        note_launch();
        k_gm_combine<<<vb, 256, 0, s>>>(V, vstride, T, n, nr, st, outer_done);
        if (e == cudaSuccess)
            e = left ? add_into(T, nrhs, X, ldx, n, nrhs, outer_done, s)
                     : apply_multiplier(G, false, T, nrhs, X, ldx, nrhs, true, outer_done, s);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cond_end(cr, s);
    }
    return e;
}

}  // namespace genp
