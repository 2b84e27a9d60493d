// genp_internal.cuh -- shared declarations of the libgenp translation units.
#pragma once

#include <utility>

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "genp.h"

namespace genp {

// ---------------------------------------------------------------------------
// Device status word of a factorization.  Non-negative doubles are kept as
// their IEEE bit patterns, which order like unsigned integers, so atomicMin /
// atomicMax on the bits give min / max of the values.
// ---------------------------------------------------------------------------
struct DevStatus {
    unsigned long long breakdown_step;   // first zero / non-finite pivot, ~0ull if none
    unsigned long long min_abs_pivot;    // bits of min |u_kk|
    unsigned long long max_abs_pivot;    // bits of max |u_kk|
    unsigned long long max_abs_u;        // bits of max |u_ij|
    unsigned long long max_abs_c;        // bits of max |c_ij| before the factorization
    int refine_iters;
    int refine_done;                     // set on the device when refinement stops
    int refine_status;                   // GENP_OK or GENP_ERR_NOCONV
    int krylov_steps;                    // GMRES steps of the last refinement (method 1)
    double anorm;                        // ||A||_inf of the last refinement
    double bwd_err[GENP_MAX_REFINE + 1];
};

constexpr int kMaxRhsChunk = 16;      // refinement works on right-hand sides in chunks

// Workspace of the refinement norms (per right-hand side).
struct DevNorms {
    unsigned long long r[kMaxRhsChunk];
    unsigned long long x[kMaxRhsChunk];
    unsigned long long b[kMaxRhsChunk];
};

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *p, double v) {
    atomicMax(p, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ void atomic_min_nonneg(unsigned long long *p, double v) {
    atomicMin(p, (unsigned long long)__double_as_longlong(v));
}

// ---------------------------------------------------------------------------
// Handles
// ---------------------------------------------------------------------------
}  // namespace genp

struct genp_multiplier {
    genp_mult_kind kind;
    int64_t n;
    int nnz;
    genp_prec grid;
    double *dense = nullptr;           // n x n (GAUSSIAN)
    float *dense_f32 = nullptr;        // n x n copy on the FP32 grid (GAUSSIAN, grid FP32/BF16)
    __nv_bfloat16 *dense_bf16 = nullptr;  // G^T, n x round8(n) (GAUSSIAN, grid BF16)
    double *g = nullptr;               // first column (CIRCULANT)
    double2 *spec = nullptr;           // DFT(g)/n in bit-reversed order (CIRCULANT, power-of-two n)
    float2 *spec_f32 = nullptr;
    double2 *twid = nullptr;           // exp(-2 pi i k / n), k < n/2
    float2 *twid_f32 = nullptr;
    int32_t *rows = nullptr;           // nnz x n (SPARSE)
    int8_t *signs = nullptr;           // nnz x n
    int32_t *inv_rows = nullptr;       // nnz x n: column whose t-th entry sits in row i
    int8_t *inv_signs = nullptr;
    int32_t *draws = nullptr;          // nnz x n Fisher-Yates draws (SPARSE)
    double scale = 1.0;
    int grid_digits = 2;               // digits of the sliced grid (dense Gaussian, grid GENP_BF16_SLICED)
    bool pm1 = false;                  // CIRCULANT_PM1 (stored as a circulant)
    bool toeplitz = false;             // TOEPLITZ (stored as a circulant of order 2n)
    int side = GENP_SIDE_RIGHT;        // C = A G (right) or C = G A (left)
    int64_t cn = 0;                    // order of the stored circulant: n, or 2n for TOEPLITZ
    int *attempt = nullptr;            // device: the draw attempt kept (CIRCULANT_PM1)
    cudaStream_t last_stream = nullptr;
};

// A recorded refinement: genp_refine's launch sequence for one set of
// arguments, replayed as one CUDA graph (see genp_refine_graphs).
struct GenpRefineGraph {
    uint64_t key[16] = {};
    cudaGraphExec_t exec = nullptr;
    uint64_t launches = 0;             // kernels the graph always runs (for genp_launch_count)
    int *body_counts = nullptr;        // device: kernels in each of its conditional bodies
};

struct genp_factors {
    GenpRefineGraph rgraph[4];         // cached refinement graphs, round robin
    int rg_next = 0;
    cudaStream_t rg_stream = nullptr;  // private stream the graphs are recorded on
    cudaStream_t rg_body[2] = {nullptr, nullptr};   // streams their nested conditional bodies are recorded on
    cudaStream_t la_stream = nullptr;  // the sliced factorization's look-ahead stream
    cudaEvent_t la_ev[2] = {nullptr, nullptr};   // update done -> block factored
    void *C = nullptr;
    int64_t n = 0, ldc = 0, nb = 64;
    genp_prec prec = GENP_FP64;
    genp::DevStatus *st = nullptr;     // device
    genp::DevNorms *norms = nullptr;   // device
    void *work = nullptr;              // device workspace for solves / refinement
    size_t work_bytes = 0;
    void *host_info = nullptr;         // pinned host copy of the status
    __nv_bfloat16 *tcA = nullptr;      // BF16 split L21 panel, n x tc_ldq (BF16 / BF16X3)
    __nv_bfloat16 *tcB = nullptr;      // BF16 split U12^T panel, n x tc_ldq
    int64_t tc_ldq = 0;
    float *qscale = nullptr;           // e4m3 tile scales of L21 and U12^T, 2 ceil(n / 128) (FP8_E4M3)
    void *W = nullptr;                 // double-float trailing matrix, n x ldw (GENP_BF16_SLICED)
    int64_t ldw = 0;
    int *exps = nullptr;               // 2n slicing exponents (GENP_BF16_SLICED)
    int nd = 0;                        // digits per operand (GENP_BF16_SLICED)
    int *trsv_sync = nullptr;          // tickets and block counters of the triangular solves
    void *trsv_y = nullptr;            // the solves' published blocks of y, n x 16 (factor type)
    void *dinv = nullptr;              // inverses of the 64 x 64 diagonal blocks of L and U (factor type)
    void *dinv_df = nullptr;           // their double-float copy, then the masked diagonal blocks (GENP_BF16_SLICED)
    bool block = false;                // block GE factors (genp_block_factor): C = L_B U_B
    cudaStream_t last_stream = nullptr;
};

namespace genp {

struct dfloat;   // dfloat.cuh

// Factors stored in FP64 (solves and refinement run in FP64).
inline bool f64_factors(genp_prec p) { return p == GENP_FP64 || p == GENP_BF16_SLICED; }

// One system of a batched solve (device array, built by genp_batched_plan).
struct BatchDesc {
    int64_t n;
    int64_t mat_off;   // offset of this system's n x n blocks (A, C, G pools), elements
    int64_t vec_off;   // offset of its n x nrhs blocks (B, X and workspace pools)
    int64_t g_off;     // offset of its circulant first column (g pool)
    int64_t sid;       // multiplier stream id (the system's index in the caller's order)
    int nb;            // CTA GEMM tile (64 or 128) chosen for its size class
    int pad;
};

// Per-system report of a batched solve.
struct BatchStatus {
    int64_t breakdown_step;
    float min_abs_pivot, max_abs_pivot, max_abs_u, max_abs_c;
    int refine_iters;
    int status;
    int escalated;     // 0; 1: inner solves switched to substitution; 2: refactored in double-float
    int krylov_steps;  // inner GMRES steps over all refinement steps
    double eta0, eta;
};

// ---------------------------------------------------------------------------
// Launchers implemented in the .cu files (all enqueue on `s`, no sync).
// ---------------------------------------------------------------------------

// Counts one kernel launch (genp_launch_count); called before every launch.
void note_launch();
void note_launches(uint64_t count);
// While a refinement is being recorded into a graph, the launch profile
// skips its launches (their events would be recorded once, not per replay).
void profile_suspend(bool on);

// rng.cu
// (grid GENP_BF16_SLICED: grid_digits balanced 7-bit digits, 1 or 2)
cudaError_t launch_make_dense(double *G, int64_t n, uint64_t seed, uint64_t stream_id, double scale,
                              genp_prec grid, float *G32, __nv_bfloat16 *Gbf, cudaStream_t s, int grid_digits = 2);
cudaError_t launch_make_circulant(double *g, int64_t n, uint64_t seed, uint64_t stream_id,
                                  double scale, genp_prec grid, cudaStream_t s);
// +-1 first column, redrawn until no DFT bin of power-of-two order vanishes
cudaError_t launch_make_circulant_pm1(double *g, int64_t n, uint64_t seed, uint64_t stream_id, int *attempt,
                                      cudaStream_t s);
cudaError_t launch_make_sparse(int32_t *rows, int8_t *signs, int32_t *inv_rows, int8_t *inv_signs,
                               int32_t *scratch, int64_t n, int nnz, uint64_t seed,
                               uint64_t stream_id, cudaStream_t s);
// G[i][j] = g[(i - j) mod cn], i, j < n
cudaError_t launch_circulant_to_dense(const double *g, int64_t cn, int64_t n, double *G, int64_t ldg,
                                      cudaStream_t s);
// Gaussian Toeplitz (2n - 1 draws) as the first column of its circulant embedding of order 2n
cudaError_t launch_make_toeplitz(double *g, int64_t n, uint64_t seed, uint64_t stream_id, double scale,
                                 genp_prec grid, cudaStream_t s);
// m x r Gaussian (or Gaussian Toeplitz) sketch of the low-rank approximation
cudaError_t launch_sketch(double *G, int64_t ldg, int64_t m, int64_t r, bool toeplitz, uint64_t seed,
                          uint64_t stream_id, double scale, cudaStream_t s);
// u = +-1 of the Householder multiplier
cudaError_t launch_make_householder(double *u, int64_t n, uint64_t seed, uint64_t stream_id, cudaStream_t s);
cudaError_t launch_batch_draw(const BatchDesc *d, int count, uint64_t seed, bool circ, float *Gpool, float *gpool,
                              cudaStream_t s);
cudaError_t launch_sparse_to_dense(const int32_t *rows, const int8_t *signs, int64_t n, int nnz,
                                   double *G, int64_t ldg, cudaStream_t s);

// gemm.cu:  D = alpha * op(A) * B + beta * Cin, row-major, op(A) = A or A^T.
// `skip` (device int, may be NULL): the kernel does nothing when *skip != 0.
template <typename T>
cudaError_t gemm(int64_t m, int64_t n, int64_t k, T alpha, const T *A, int64_t lda, bool transA,
                 const T *B, int64_t ldb, T beta, const T *Cin, int64_t ldci, T *D, int64_t ldd,
                 const int *skip, cudaStream_t s);

// circ.cu: circulant products through the DFT (Thm. 2.1).
bool circ_fft_supported(int64_t n);
cudaError_t circ_prepare(genp_multiplier *G, cudaStream_t s);
// out_p = ifft(fft(in_p) * H) for `count` vectors of length n: element i of
// vector p at in[p*pstride + i*estride].  mode 0: H = conj(spec) (v G);
// mode 1: H = spec (G v); mode 2: H = conj(spec) (G^T v).
template <typename TI, typename TO>
cudaError_t circ_apply(const genp_multiplier *G, int mode, const TI *in, int64_t in_pstride,
                       int64_t in_estride, TO *out, int64_t out_pstride, int64_t out_estride,
                       int64_t count, const int *skip, cudaStream_t s);
// X (+)= G Y (trans false) or G^T Y on the columns of Y (n x nrhs double).
cudaError_t circ_apply_cols(const genp_multiplier *G, bool trans, const double *Y, int64_t ldy, double *X,
                            int64_t ldx, int64_t nrhs, bool accumulate, const int *skip, cudaStream_t s);
// Direct (non-FFT) C = A * G in 2n^3 operations, G the leading n x n block of
// the circulant of order cn with first column g (cn = n circulant, 2n Toeplitz).
template <typename TI, typename TO>
cudaError_t circ_matmul_direct(const double *g, int64_t cn, int64_t n, const TI *A, int64_t lda, TO *C,
                               int64_t ldc, cudaStream_t s);

cudaError_t circ_apply_direct(const double *g, int64_t cn, int64_t n, bool trans, const double *Y, int64_t ldy,
                              double *X, int64_t ldx, int64_t nrhs, bool accumulate, const int *skip, cudaStream_t s);

// house.cu: the Householder multiplier H = I - 2 u u^T / n (u = +-1)
template <typename TI, typename TO>
cudaError_t house_precondition(const genp_multiplier *G, const TI *A, int64_t lda, TO *C, int64_t ldc,
                               cudaStream_t s);
cudaError_t house_apply(const genp_multiplier *G, const double *Y, int64_t ldy, double *X, int64_t ldx,
                        int64_t nrhs, bool accumulate, const int *skip, cudaStream_t s);
cudaError_t house_to_dense(const genp_multiplier *G, double *D, int64_t ldd, cudaStream_t s);

// sparse.cu
template <typename TI, typename TO>
cudaError_t sparse_precondition(const genp_multiplier *G, const TI *A, int64_t lda, TO *C, int64_t ldc,
                                cudaStream_t s);
// X = G Y (trans = false) or G^T Y, X and Y n x nrhs double; accumulate: X += ...
cudaError_t sparse_apply(const genp_multiplier *G, bool trans, const double *Y, int64_t ldy, double *X,
                         int64_t ldx, int64_t nrhs, bool accumulate, const int *skip, cudaStream_t s);

// gemm_tc.cu: D = alpha * A * Bt^T + beta * Cin on the tensor cores (BF16 in, FP32 out).
cudaError_t tc_gemm_bf16(int64_t m, int64_t n, int64_t K, float alpha, const __nv_bfloat16 *A, int64_t lda,
                         const __nv_bfloat16 *Bt, int64_t ldb, float beta, const float *Cin, int64_t ldci, float *D,
                         int64_t ldd, const int *skip, cudaStream_t s);
// gemm_tc.cu: D = alpha * sum_kt scA[tm][kt] scB[tn][kt] A_kt Bt_kt^T + beta * Cin on
// the tensor cores, A (m x K) and Bt (n x K) e4m3 codes with one scale per
// 128 x 128 tile (nkt = ceil(K / 128) per tile row), FP32 out.
cudaError_t tc_gemm_e4m3(int64_t m, int64_t n, int64_t K, float alpha, const uint8_t *A, int64_t lda, const float *scA,
                         const uint8_t *Bt, int64_t ldb, const float *scB, float beta, const float *Cin, int64_t ldci,
                         float *D, int64_t ldd, cudaStream_t s);
// mixed.cu: e4m3 codes of X (m x K; X = src, or src^T when trans, src then
// K x m) with a power-of-two scale per 128 x 128 tile, scales[ti nkt + kt].
template <typename T>
cudaError_t quant_e4m3(const T *src, int64_t lds, int64_t m, int64_t K, bool trans, uint8_t *dst, int64_t ldq,
                       float *scales, cudaStream_t s);
int64_t e4m3_tiles(int64_t rows, int64_t K);
// Reads the device-side timeout flag of the tensor-core kernels (synchronizes).
int tc_timeout_flag(bool reset);
// CUDA-event timing of the sliced tensor-core launches (genp_profile_*).
void tc_profile_enable(bool on);
int tc_profile_read(double *ms, double *flops);
int tc_profile_launches(double *ms, double *flops, int cap);
// The other kernel classes of the launch profile, each launch with its
// algorithmic work (bytes for the HBM-bound classes, flops otherwise).
enum ProfClass {
    kProfTensor = 0, kProfTrsv = 1, kProfGemv = 2, kProfFactorAux = 3, kProfOuter = 4, kProfPrecond = 5,
    kProfClasses = 6
};
// Events around one launch of class c, or nullptr when profiling is off.
std::pair<cudaEvent_t, cudaEvent_t> *profile_class_slot(int c, double work);
// Sum of the recorded launches of class c (synchronizes on their events);
// the work of launches that found their skip flag set is left out.
int profile_class_read(int c, double *ms, double *work);
// Launches of the triangular solves / matrix-vector products that returned
// at once on their skip flag (device counters; reset on request).
unsigned int trsv_skipped_count(bool reset);
unsigned int gemv_skipped_count(bool reset);
// Records the start / end event of a launch when ev is not null.
inline void prof_begin(std::pair<cudaEvent_t, cudaEvent_t> *ev, cudaStream_t s) {
    if (ev) cudaEventRecord(ev->first, s);
}
inline void prof_end(std::pair<cudaEvent_t, cudaEvent_t> *ev, cudaStream_t s) {
    if (ev) cudaEventRecord(ev->second, s);
}
// D += alpha * A B on the tensor cores with FP64-class accuracy, from the
// nd-digit slices of sliced.cu: Aq (m x nd kpad) and Bq (n x nd kpad, B
// transposed) with their row / column exponents ea, fb.
// D is double-float.  alpha must be a power of two (it is applied to both
// halves of each sum).  kpad <= kSlicedChunk.
// The same with nda digits of A and ndb of B (nda = ndb = 3 .. 7, or
// nda = 2 and ndb = 5 .. 7): pairs with t + u <= max(nda, ndb) - 1.
cudaError_t tc_gemm_sliced2(int nda, int ndb, int64_t m, int64_t n, int64_t kpad, float alpha,
                            const __nv_bfloat16 *Aq, int64_t lda, const __nv_bfloat16 *Bq, int64_t ldb, const int *ea,
                            const int *fb, dfloat *D, int64_t ldd, cudaStream_t s);
cudaError_t tc_gemm_sliced(int nd, int64_t m, int64_t n, int64_t kpad, float alpha, const __nv_bfloat16 *Aq,
                           int64_t lda, const __nv_bfloat16 *Bq, int64_t ldb, const int *ea, const int *fb, dfloat *D,
                           int64_t ldd, cudaStream_t s);
// SMs the persistent sliced product leaves free from now on in this host
// thread (0: none); returns the previous value.
int sliced_spare_sms(int k);

// sliced.cu: exact 7-bit digit slicing of FP64 operands (Ozaki scheme).
int64_t sliced_kpad(int64_t K);   // K rounded up to the k-tile
int sliced_slices(int nd);        // digit slices per operand (operand width slices * kpad)
int sliced_digits();              // digits of the GENP_BF16_SLICED path
int set_sliced_digits(int nd);    // returns the previous value, -1 if nd is unsupported
int sliced_precond_digits();      // digits of the sliced C = A G
int set_sliced_precond_digits(int nd);
int sliced_mult_digits();         // digits of a new dense Gaussian's sliced grid (1 or 2)
int set_sliced_mult_digits(int d);   // returns the previous value, -1 if d is not 1 or 2
// rows of src (m x K): dst[i][p*kpad + k] = slice p of src[i][k] 2^-q_k
// (kkey null: no scaling; else q_k from kkey[k], see sliced_inner_exps);
// exps[i] = row exponent
cudaError_t slice_rows(int nd, const double *src, int64_t lds, int64_t m, int64_t K, __nv_bfloat16 *dst, int64_t ldq,
                       int *exps, cudaStream_t s, const unsigned long long *kkey = nullptr);
// columns of src (K x n), written transposed: dst[j][p*kpad + k] = slice p of
// src[k][j] 2^+q_k (kkey may be null); exps[j] = column exponent
cudaError_t slice_cols_T(int nd, const double *src, int64_t lds, int64_t K, int64_t n, __nv_bfloat16 *dst,
                         int64_t ldq, int *exps, cudaStream_t s, const unsigned long long *kkey = nullptr);
// keys[k] of max_i |L[i][k]| over the m x K block L, from which the slicing
// kernels take q_k = e with max_i |L[i][k]| < 2^e: the power-of-two scaling
// of the inner dimension of L U that balances the columns of L (and,
// inversely, the rows of U) before slicing
cudaError_t sliced_inner_exps(const double *L, int64_t ldl, int64_t m, int64_t K, unsigned long long *keys,
                              cudaStream_t s);
// the same three from the double-float trailing matrix (each entry taken
// exactly as FP64), so a block needs no FP64 copy before it is sliced
cudaError_t slice_rows(int nd, const dfloat *src, int64_t lds, int64_t m, int64_t K, __nv_bfloat16 *dst, int64_t ldq,
                       int *exps, cudaStream_t s, const unsigned long long *kkey);
cudaError_t slice_cols_T(int nd, const dfloat *src, int64_t lds, int64_t K, int64_t n, __nv_bfloat16 *dst,
                         int64_t ldq, int *exps, cudaStream_t s, const unsigned long long *kkey);
cudaError_t sliced_inner_exps(const dfloat *L, int64_t ldl, int64_t m, int64_t K, unsigned long long *keys,
                              cudaStream_t s);
// double <-> double-float copies of an m x n block
// (with amax: max |src| into that status word as well)
cudaError_t df_from_f64(const double *src, int64_t lds, dfloat *dst, int64_t ldd, int64_t m, int64_t n,
                        cudaStream_t s, unsigned long long *amax = nullptr);
cudaError_t df_to_f64(const dfloat *src, int64_t lds, double *dst, int64_t ldd, int64_t m, int64_t n,
                      cudaStream_t s);
// D = alpha * W + beta * D (W double-float, D double; beta == 0 ignores D)
cudaError_t df_axpby(double alpha, const dfloat *W, int64_t ldw, double beta, double *D, int64_t ldd, int64_t m,
                     int64_t n, cudaStream_t s);
// D (double-float, m x n) = A B, A m x K and B K x n FP64, K cut in chunks of
// at most kSlicedChunk (kSlicedChunk2 for a one- or two-digit A side); Aq, Bq hold
// (m or n) x nd chunk BF16, exps m + n ints.
// Dt (double-float, n x m) = (A B)^T = B^T A^T, with B's columns (ndb
// digits) on the M side and A's rows (nda digits) on the N side: for a B
// exact in few digits (a multiplier on the sliced grid) the wide operand
// then sits along N, where one MMA covers several of its digits.
// Bq holds n x ndb chunk, Aq m x nda chunk BF16 (chunk kSlicedChunk2 for
// ndb <= 2, else kSlicedChunk); exps n + m ints.
cudaError_t sliced_matmul_t(int nda, int ndb, int64_t m, int64_t n, int64_t K, const double *A, int64_t lda,
                            const double *B, int64_t ldb, dfloat *Dt, int64_t lddt, __nv_bfloat16 *Bq,
                            __nv_bfloat16 *Aq, int *exps, cudaStream_t s);
// dst (m x n, FP64) = src^T, src n x m double-float
cudaError_t df_to_f64_T(const dfloat *src, int64_t lds, double *dst, int64_t ldd, int64_t m, int64_t n,
                        cudaStream_t s);
cudaError_t sliced_matmul(int nd, int64_t m, int64_t n, int64_t K, const double *A, int64_t lda, const double *B,
                          int64_t ldb, dfloat *D, int64_t ldd, __nv_bfloat16 *Aq, __nv_bfloat16 *Bq, int *exps,
                          cudaStream_t s, int ndb = 0);
constexpr int kSlicedOuter = 512;       // outer step (Schur update K) of the sliced factorization
constexpr int64_t kSlicedChunk = 512;   // keeps the digit groups of weight >= 2^-49 exact in FP32
// With a two-digit M side (a multiplier on the sliced grid) a group holds at
// most two pairs of |d_t d_u| <= 2^13 (one pair of 2^14 for group 0), and
// with a one-digit side one pair of at most 2^14, so every group but the
// last stays exact in FP32 up to K = 1024.
constexpr int64_t kSlicedChunk2 = 1024;
constexpr int64_t kSlicedLdq = 7 * kSlicedChunk;    // operand width for up to 7 digits

// mixed.cu: BF16 split operands.  terms = 1 (GENP_BF16) or 6 (GENP_BF16X3).
int split_terms(genp_prec p);
// dst[i][b*k + kk] = term_b(src[i][kk]) for the left operand (left = true) or
// the right operand's term order; single_term >= 0 writes that one term only.
template <typename T>
cudaError_t split_rows(const T *src, int64_t lds, int64_t m, int64_t k, __nv_bfloat16 *dst, int64_t ldq, int terms,
                       bool left, int single_term, cudaStream_t s);
// dst[j][b*k + kk] = term_b(src[kk][j]) (right operand, transposed to K-major).
template <typename T>
cudaError_t split_cols_T(const T *src, int64_t lds, int64_t k, int64_t m, __nv_bfloat16 *dst, int64_t ldq, int terms,
                         cudaStream_t s);
__host__ __device__ inline int64_t round8(int64_t x) { return (x + 7) / 8 * 8; }

// Krylov steps per inner GMRES solve of the batched kernel.
constexpr int kBatchedKrylov = 16;

// Arguments of the batched kernels (batched.cu, batched_impl.cuh).
struct BatchedArgs {
    const BatchDesc *desc;
    int count;
    int *counter;         // work queue (reset before each launch)
    const void *A;        // A pool, FP64 (a64) or FP32
    int a64;
    const double *B;      // right-hand sides (forward)
    double *X;            // solutions (forward output; adjoint input)
    float *C;             // factors, A-pool layout
    const float *G, *g;   // dense multipliers or circulant first columns
    float *scratch;       // per-CTA scratch, `stride` floats each
    int64_t stride;
    int nmax, nr, circ, max_iter;
    double tol;
    BatchStatus *stat;
    const double *gX;     // adjoint: incoming gradient
    double *L, *dB;       // adjoint: Lambda (vector-pool layout), dB (may be null)
    float *dA;            // adjoint: dA (A-pool layout, may be null)
    unsigned long long *prof;   // optional: per-CTA SM cycles by phase (kBatchedPhases each)
};
// Phases of the batched kernel's cycle profile: C = A G, factorization,
// inverses of the factors, first solve and x = G y, FP64 residuals, inner
// GMRES, x += G d.
constexpr int kBatchedPhases = 7;
// batched.cu (nmax: largest order of the batch; nr: right-hand sides)
int batched_blocks_per_sm(int nr, int nmax);
// Floats of scratch each persistent CTA needs.
int64_t batched_scratch_stride(int nr, int nmax);
cudaError_t launch_batched(BatchedArgs a, int grid, cudaStream_t s);
cudaError_t launch_batched_adjoint(BatchedArgs a, int grid, cudaStream_t s);
// per right-hand-side class NR in {1, 2, 4, 8, 16} (batched_r*.cu)
#define GENP_BATCHED_DECL(NR)                                                  \
    int batched_blocks_per_sm_r##NR(int nmax);                                 \
    cudaError_t batched_launch_r##NR(const BatchedArgs &a, int grid, cudaStream_t s); \
    cudaError_t batched_adjoint_r##NR(const BatchedArgs &a, int grid, cudaStream_t s);
GENP_BATCHED_DECL(1)
GENP_BATCHED_DECL(2)
GENP_BATCHED_DECL(4)
GENP_BATCHED_DECL(8)
GENP_BATCHED_DECL(16)
#undef GENP_BATCHED_DECL
// batched_escalate.cu (systems whose status is not GENP_OK after launch_batched)
int batched_escalate_blocks_per_sm();
// Doubles of double-float scratch each persistent CTA of the escalation needs.
int64_t batched_escalate_stride();
cudaError_t launch_batched_escalate(const BatchDesc *d, int count, int *counter, const void *Apool, bool a_f64,
                                    const double *Bpool, double *Xpool, const float *Gpool, const float *gpool,
                                    double *Rpool, double *scratch64, int nr, bool circ, int max_iter, double tol,
                                    BatchStatus *stat, int grid, cudaStream_t s);

// lu.cu
cudaError_t factor_run(genp_factors *F, cudaStream_t s);
cudaError_t status_reset(genp_factors *F, cudaStream_t s);

// lowrank.cu: randomized low-rank approximation (Proto-Alg. 5.1)
cudaError_t lowrank_run(int64_t m, int64_t n, const double *A, int64_t lda, int64_t r, bool toeplitz, uint64_t seed,
                        uint64_t sid, double *G, int64_t ldg, double *Q, int64_t ldq, double *R, int64_t ldr,
                        double *AQ, int64_t ldaq, int *fail, void *work, cudaStream_t s);
size_t lowrank_work_bytes(int64_t m, int64_t n, int64_t r);
cudaError_t numerical_rank_run(int64_t m, int64_t n, const double *A, int64_t lda, int64_t r_lo, int64_t r_hi,
                               double cond_max, uint64_t seed, uint64_t sid, int64_t *rank, double *B, int64_t ldb,
                               void *work, double *host_kappa, cudaStream_t s);
size_t numerical_rank_work_bytes(int64_t m, int64_t n, int64_t r_hi);

// solve.cu
// Y <- U^{-1} L^{-1} Y in the factor's precision, Y n x nrhs of type T
template <typename T>
cudaError_t lu_solve_inplace(const genp_factors *F, T *Y, int64_t ldy, int64_t nrhs, bool transposed,
                             const int *skip, cudaStream_t s);
template <typename TS, typename TD>
cudaError_t convert_matrix(const TS *src, int64_t lds, TD *dst, int64_t ldd, int64_t m, int64_t n,
                           const int *skip, cudaStream_t s);
cudaError_t refine_init(genp_factors *F, const double *A, int64_t lda, int64_t n, cudaStream_t s);
cudaError_t refine_check(genp_factors *F, const double *R, int64_t ldr, const double *X, int64_t ldx,
                         const double *B, int64_t ldb, int64_t n, int64_t nrhs, int it, double tol,
                         int max_iter, int last_chunk, cudaStream_t s);
// Reads the device-side timeout flag of the triangular solves (synchronizes).
int solve_timeout_flag(bool reset);
// ints of synchronization state a triangular solve of order n needs
int64_t trsv_sync_ints(int64_t n);
int64_t trsv_y_elems(int64_t n);
// elements of F->dinv, and its computation (after every factorization)
int64_t diag_inverse_elems(int64_t n);
// gemm_tc.cu: 2-D tensor map (TMA) of a rows x cols row-major matrix of
// 8-byte elements (FP64, or double-float pairs), leading dimension ld, for
// boxes of box_rows x box_cols, no swizzle; elements past rows or cols read
// as zero.  False when the driver cannot encode it (ptr and ld * 8 must be
// 16-byte aligned, box_cols * 8 a multiple of 16, both box sides <= 256).
bool make_map_8b(CUtensorMap *map, const void *ptr, int64_t rows, int64_t cols, int64_t ld, int box_cols,
                 int box_rows);
cudaError_t invert_diag_blocks(genp_factors *F, cudaStream_t s);
// block.cu: block Gaussian elimination of F->C with explicit pivot-block
// inverses (nb = 64), the inverses written to F->dinv.
cudaError_t factor_block(genp_factors *F, cudaStream_t s);
// lu.cu: max |c_ij| of an n x n FP64 matrix into the status word *out.
cudaError_t maxabs_f64(const double *C, int64_t n, int64_t ldc, unsigned long long *out, cudaStream_t s);
cudaError_t outer_update(const double *Lam, int64_t ldl, const double *X, int64_t ldx, int64_t n,
                         int64_t nrhs, void *dA, int64_t ldda, bool dA_f32, cudaStream_t s);

// Conditional bodies of a recorded refinement graph.  A step that a
// converged refinement no longer needs (a residual check, a correction, a
// Krylov step) is recorded as the body of an IF node, whose condition a
// one-thread kernel sets from the step's done flag just before it, so the
// replayed graph skips it instead of launching kernels that return at once.
// cond_begin opens a body (s then names the stream it is recorded on) and
// cond_end closes it; both do nothing when c is null (launches enqueued as
// they are).  api.cu.
struct CondRec;
cudaError_t cond_begin(CondRec *c, cudaStream_t &s, const int *done);
cudaError_t cond_end(CondRec *c, cudaStream_t &s);

// gmres.cu: GMRES-IR (genp_refine method 1); work holds gmres_work_bytes(n, nrhs)
size_t gmres_work_bytes(int64_t n, int64_t nrhs);
cudaError_t refine_gmres(genp_factors *F, const genp_multiplier *G, const double *A, int64_t lda, const double *B,
                         int64_t ldb, int64_t nrhs, double *X, int64_t ldx, double tol, int max_iter, void *work,
                         cudaStream_t s, CondRec *cr = nullptr);

// api.cu helpers
// X[r][c] += Y[r][c] (n x nr), skipped when *skip != 0
cudaError_t add_into(const double *Y, int64_t ldy, double *X, int64_t ldx, int64_t n, int64_t nr, const int *skip,
                     cudaStream_t s);
cudaError_t apply_multiplier(const genp_multiplier *G, bool trans, const double *Y, int64_t ldy,
                             double *X, int64_t ldx, int64_t nrhs, bool accumulate, const int *skip,
                             cudaStream_t s);

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace genp
