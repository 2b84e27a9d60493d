/*
 * genp.h -- C ABI of libgenp: Gaussian elimination with no pivoting made
 * numerically safe by a random multiplier, on one GB300 (sm_103a) GPU.
 *
 * The method (Pan & Qian, "More on the Power of Randomized Matrix
 * Multiplication", Sec. 1.1 and Cor. 4.1): to solve A x = b for a
 * nonsingular, well conditioned A whose leading blocks may be singular or
 * ill conditioned, draw a random multiplier G, form C = A G, factor C = L U
 * by GENP (no row or column interchange), solve L U y = b and return
 * x = G y (so A x = A G y = C y = b).  Theorem 4.1 (the MH form with M = A,
 * H = G) and Corollary 4.1 bound the conditioning of C and of all of its
 * leading blocks in terms of that of A; Theorem 2.2 then bounds every pivot.
 *
 * Conventions for every entry point:
 *  - Matrices are row-major with an explicit leading dimension (element
 *    (i, j) of X lives at X[i*ldx + j]); ld >= number of columns.
 *  - Every matrix/vector pointer is a DEVICE pointer owned by the caller
 *    (the library never frees it and keeps no reference past the call,
 *    except genp_factors, which refers to the caller's C buffer until it is
 *    destroyed or refactored).
 *  - `cuda_stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls only enqueue work on that stream and return; they do
 *    not synchronize, except genp_info_fetch and the *_destroy calls.
 *  - Argument errors are detected on the host and returned at once
 *    (GENP_ERR_ARG) with nothing enqueued.  Conditions found on the device
 *    (a zero or non-finite pivot, refinement that does not converge) are
 *    written to a status word inside the factors handle and reported by
 *    genp_info_fetch.  The library never aborts the process and its kernels
 *    never trap.
 *  - Handles are opaque and library-owned; a handle may be used from one
 *    stream at a time.
 *  - Calls that document a cudaMallocAsync workspace take it from the
 *    device's default memory pool; on first use per device the library
 *    raises that pool's release threshold so freed workspace stays mapped
 *    for the next call (the setting belongs to this process's pool).
 */
#ifndef GENP_H
#define GENP_H

#include <stdint.h>

#if defined(__GNUC__)
#define GENP_API __attribute__((visibility("default")))
#else
#define GENP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GENP_OK = 0,
    GENP_ERR_ARG = -1,         /* invalid argument; nothing was enqueued            */
    GENP_ERR_BREAKDOWN = -2,   /* GENP met a zero or non-finite pivot (Sec. 1.1)    */
    GENP_ERR_NOCONV = -3,      /* refinement stopped above the requested tolerance */
    GENP_ERR_CUDA = -4,        /* a CUDA runtime call failed                        */
    GENP_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up                */
    GENP_ERR_NOMEM = -6,       /* device memory could not be allocated              */
    GENP_ERR_UNSUPPORTED = -7  /* valid combination that the library does not offer*/
} genp_status;

/* Random multiplier families.
 *  GAUSSIAN:    dense G with iid N(0, scale^2) entries (Definition 3.2,
 *               the set G_{0,scale}^{n x n}).
 *  CIRCULANT:   G[i][j] = g[(i - j) mod n] with iid N(0, scale^2) first
 *               column g (Sec. 2.3 and Definition 3.2, Z_{0,scale}).
 *  SPARSE_PM1:  G = sum_{t < nnz} D_t P_t, P_t independent uniform random
 *               permutation matrices, D_t random +-1 diagonals, so every
 *               column and every row holds nnz signed unit entries
 *               (coinciding positions add).  The paper names sparse
 *               multipliers (Sec. 1 and Sec. 8) without fixing a structure;
 *               this is the structure the library uses.
 *  CIRCULANT_PM1: circulant whose first column holds random signs +-1, the
 *               multipliers of the paper's tests (Sec. 7.1, Table 7.1).
 *               Such a circulant is exactly singular when a DFT bin of g
 *               vanishes (probability about 0.18 at n = 64); draws are
 *               repeated (attempt a = 0, 1, ... on the Philox counter) until
 *               no bin of power-of-two order vanishes, an exact integer test
 *               (the sum of g, and the folded sums for every x^m + 1 with
 *               2m | n), complete when n is a power of two.  scale ignored.
 *  IDENTITY:    G = I, i.e. plain GENP of A (no preconditioning), the
 *               paper's comparison point; seed, scale and grid ignored.
 *  TOEPLITZ:    G[i][j] = t_{i-j} with 2n - 1 iid N(0, scale^2) entries
 *               t_{-(n-1)} .. t_{n-1} (Definition 3.2, T_{0,scale}).  Stored
 *               as the first column of the circulant of order 2n whose
 *               leading n x n block is G; products run through its DFT
 *               (n <= 4096) or directly.
 *  HOUSEHOLDER_PM1: G = I - 2 u u^T / n with u of random signs +-1, the
 *               Householder multipliers of the tests cited in Sec. 7.1.  The
 *               printed form I - u v^T / u^T v is a projection (singular);
 *               this is the orthogonal reflector.  A rank-one change of A:
 *               it repairs leading blocks whose rank falls short by one, not
 *               more.  scale and grid ignored (its entries 1 - 2/n and +-2/n
 *               are exact in FP32 when n is a power of two). */
typedef enum {
    GENP_MULT_GAUSSIAN = 0,
    GENP_MULT_CIRCULANT = 1,
    GENP_MULT_SPARSE_PM1 = 2,
    GENP_MULT_CIRCULANT_PM1 = 3,
    GENP_MULT_IDENTITY = 4,
    GENP_MULT_TOEPLITZ = 5,
    GENP_MULT_HOUSEHOLDER_PM1 = 6
} genp_mult_kind;

/* Arithmetic of a factorization.
 *  FP64: C and the factors are double; every step in FP64.
 *  FP32: C and the factors are float; every step in FP32.
 *  BF16: C and the factors are stored as float (the master copy); the
 *        Schur-complement products use BF16 operands on the tensor cores
 *        with FP32 accumulation; the diagonal blocks are factored in
 *        double-float arithmetic (48 bits: FP64-class pivots).
 *  FP8_E4M3: as BF16 with e4m3 operands (3 mantissa bits) and one
 *        power-of-two scale per 128 x 128 operand tile (genp_quantize_e4m3);
 *        for a Gaussian multiplier A G runs on the e4m3 tensor cores too,
 *        with G drawn on the FP8 grid (value_grid GENP_FP8_E4M3).  The
 *        factors carry errors of order 2^-4 times the element growth: they
 *        precondition GMRES-IR on well-conditioned systems of moderate
 *        growth and fail to where that product approaches 1.
 *  BF16X3: as BF16, but every operand is split into three BF16 terms and
 *        six of their products are accumulated (a1b1 + a1b2 + a2b1 + a1b3 +
 *        a2b2 + a3b1), which brings the tensor-core products close to FP32
 *        accuracy at six times the BF16 work.
 *  BF16_SLICED: C and the factors are double, as for FP64; the diagonal
 *        blocks and the block row and column are solved in double-float
 *        arithmetic (48 bits, on the FP32 pipe), while the Schur-complement
 *        products (and, for a Gaussian multiplier, A G) run on the BF16
 *        tensor cores: each FP64 operand row / column gets a
 *        power-of-two scale and is cut into 5, 6 or 7 exact 7-bit digits
 *        (genp_sliced_digits; A G takes genp_sliced_precondition_digits),
 *        and the digit products of the leading
 *        weights are accumulated in FP32, all but the smallest weight group
 *        exactly (Ozaki, Ogita, Oishi and Rump's error-free splitting).  With
 *        7 digits the products carry about 46 correct bits against the
 *        operands' scales; the trailing matrix is held as double-float pairs
 *        (48 bits) between steps.  The diagonal blocks and block rows and
 *        columns are solved nb wide; the tensor-core updates take outer
 *        blocks of max(2 nb, 512) and, inside them, the inner blocks'
 *        updates (the inner dimension of every update balanced by powers of
 *        two).  FP64 refinement (GMRES-IR at large growth) takes the solve
 *        to FP64 accuracy. */
typedef enum {
    GENP_FP64 = 0,
    GENP_FP32 = 1,
    GENP_BF16 = 2,
    GENP_FP8_E4M3 = 3,
    GENP_BF16X3 = 4,
    GENP_BF16_SLICED = 5
} genp_prec;

typedef struct genp_multiplier genp_multiplier;
typedef struct genp_factors genp_factors;

#define GENP_MAX_REFINE 32
#define GENP_GMRES_RESTART 30

/* Host-side report filled by genp_info_fetch. */
typedef struct {
    int32_t status;              /* GENP_OK, GENP_ERR_BREAKDOWN or GENP_ERR_NOCONV       */
    int32_t refine_iters;        /* refinement steps taken by the last genp_refine      */
    int64_t breakdown_step;      /* first step with a zero / non-finite pivot, else -1  */
    double min_abs_pivot;        /* min_k |u_kk|                                         */
    double max_abs_pivot;        /* max_k |u_kk|                                         */
    double growth;               /* max|U| / max|C|                                      */
    double bwd_err[GENP_MAX_REFINE + 1]; /* backward error before refinement and after  */
                                 /* each step of the last genp_refine (see genp_refine) */
    int32_t krylov_steps;        /* GMRES steps (Krylov vectors) of the last genp_refine */
    int32_t reserved;
} genp_info;

/* Library version string, e.g. "genp 0.1 sm_103a". */
GENP_API const char *genp_version(void);

/* Human-readable name of a status code. */
GENP_API const char *genp_status_string(genp_status s);

/* Draws a random multiplier from a counter-based generator (Philox4x64-10,
 * key = (seed, stream_id)); the same (kind, n, seed, stream_id, scale,
 * nnz_per_col, value_grid) always yields the same G bit for bit.
 *  kind        GENP_MULT_*.
 *  n           order of G, 1 <= n <= 2^31 - 1 (dense: n*n*8 bytes of storage).
 *  scale       standard deviation of the Gaussian entries (Gaussian and
 *              circulant; e.g. 1/sqrt(n) for variance 1/n); ignored for SPARSE.
 *  nnz_per_col signed entries per column for SPARSE (1..16); ignored otherwise.
 *  value_grid  GENP_FP64: entries as drawn.  GENP_BF16: every entry rounded
 *              to the nearest BF16 value (Thm. 4.1 allows a perturbed
 *              Gaussian H = H' + V), so the tensor-core product and the FP64
 *              correction x += G d use exactly the same G.  GENP_FP32:
 *              drawn in single precision.  GENP_FP8_E4M3: the single
 *              precision draw rounded to an e4m3 value times 2^e, one e for
 *              the matrix (the least with 12.5 scale <= 448 2^e, so no entry
 *              saturates).  GENP_BF16_SLICED: the single precision draw
 *              (as for GENP_FP32) rounded to the
 *              nearest integer multiple of 2^(E - 13), ties to even, with E
 *              the least integer such that 12.5 scale <= 2^E: every entry
 *              then holds two exact 7-bit digits at any column scale, so
 *              the sliced C = A G (c_prec GENP_BF16_SLICED) forms 13 digit
 *              products instead of 28 at the same accuracy, and
 *              x += G d uses that same G.  The rounding moves an entry by at
 *              most 2^(E - 14) < 1.6e-3 scale, a perturbed Gaussian that
 *              Thm. 4.1 covers (G = G' + U).  A dense Gaussian takes the
 *              grid of genp_sliced_multiplier_digits at its creation: with
 *              one digit (the default) the multiples are of 2^(E - 6), an
 *              entry moves by at most 2^(E - 7) (about 0.1 to 0.2 of the
 *              scale), and A G forms 5 digit products for five digits of A
 *              (7 for seven).  SPARSE, IDENTITY and HOUSEHOLDER_PM1 ignore
 *              it.
 *  out         receives the handle; the library owns G's device storage.
 * Errors: GENP_ERR_ARG, GENP_ERR_NOMEM, GENP_ERR_CUDA. */
GENP_API genp_status genp_make_multiplier(genp_mult_kind kind, int64_t n, uint64_t seed, uint64_t stream_id,
                                 double scale, int nnz_per_col, genp_prec value_grid,
                                 void *cuda_stream, genp_multiplier **out);

/* Side of the multiplier (Thm. 4.1 and Cor. 4.1 cover both products GM
 * and MH).
 *  GENP_SIDE_RIGHT (the default): genp_precondition forms C = A G and
 *      genp_solve returns X = G U^{-1} L^{-1} B.
 *  GENP_SIDE_LEFT: C = G A and X = U^{-1} L^{-1} (G B); genp_refine takes
 *      steps d = U^{-1} L^{-1} (G r), x += d (GMRES-IR on G A d = G r), and
 *      genp_adjoint returns Lambda = A^{-T} gX = G^T L^{-T} U^{-T} gX.
 * The left side is offered with A in FP64 and FP64, FP32 or BF16_SLICED
 * factorizations (genp_precondition returns GENP_ERR_UNSUPPORTED for BF16
 * and BF16X3).  Set the side before genp_precondition and keep it for the
 * solves of the same factors.
 *  side   GENP_SIDE_RIGHT or GENP_SIDE_LEFT sets it; -1 only queries.
 * Returns the previous side, or GENP_ERR_ARG for a NULL G or another side. */
typedef enum { GENP_SIDE_RIGHT = 0, GENP_SIDE_LEFT = 1 } genp_side;
GENP_API int genp_multiplier_side(genp_multiplier *G, int side);

/* Redraws G in place with a new (seed, stream_id), keeping kind, n, scale,
 * nnz and grid; allocates nothing, so it may run inside a timed or captured
 * region.  This is the paper's recovery rule too (Sec. 5, Remark B.1): on a
 * failure, apply the method again with fresh random parameters.
 * The result equals genp_make_multiplier with the new seed bit for bit.
 * Errors: GENP_ERR_ARG, GENP_ERR_CUDA. */
GENP_API genp_status genp_redraw_multiplier(genp_multiplier *G, uint64_t seed, uint64_t stream_id,
                                            void *cuda_stream);

/* Copies G's description into caller device buffers (any may be NULL):
 *  dense      n x n (ld ldd) double: the full matrix G (every kind).
 *  first_col  n doubles: g (CIRCULANT, CIRCULANT_PM1); for TOEPLITZ 2n
 *             doubles: the first column of its circulant embedding,
 *             t_0 .. t_{n-1}, 0, t_{-(n-1)} .. t_{-1}; for HOUSEHOLDER_PM1
 *             n doubles: u.
 *  rows       nnz*n int32: row of the t-th entry of column j at [t*n + j] (SPARSE).
 *  signs      nnz*n int8: its sign (SPARSE). */
GENP_API genp_status genp_multiplier_export(const genp_multiplier *G, double *dense, int64_t ldd,
                                   double *first_col, int32_t *rows, int8_t *signs,
                                   void *cuda_stream);

/* Order, kind and nnz of a multiplier (host-side, no device work). */
GENP_API genp_status genp_multiplier_query(const genp_multiplier *G, int64_t *n, int *kind, int *nnz_per_col);

/* Frees G (cudaFree waits for work still using it). NULL is ignored. */
GENP_API void genp_multiplier_destroy(genp_multiplier *G);

/* C = A G  (Thm. 4.1, the MH product; Cor. 4.1).
 *  A      n x n, ld lda; double if a_prec == GENP_FP64, float if GENP_FP32.
 *  C      n x n, ld ldc; double if c_prec is GENP_FP64 or GENP_BF16_SLICED,
 *         else float.  C must not overlap A.
 *  c_prec the factorization the product is for: FP64 (DFMA), FP32 (FFMA),
 *         BF16 (tensor cores, A rounded to BF16, G must have value_grid BF16),
 *         FP8_E4M3 (tensor cores, A as tile-scaled e4m3 codes, G must have
 *         value_grid FP8_E4M3),
 *         BF16_SLICED (A double; a dense G on the tensor cores by digit
 *         slicing, in K chunks of 512, genp_sliced_precondition_digits
 *         digits; other kinds as FP64).
 * Dense G costs 2n^3 flops; a circulant G is applied by FFT in
 * O(n^2 log n) (Thm. 2.1) when n is a power of two <= 8192; the sparse G is
 * a signed gather of nnz columns per output column. */
GENP_API genp_status genp_precondition(const genp_multiplier *G, const void *A, int64_t lda, genp_prec a_prec,
                              void *C, int64_t ldc, genp_prec c_prec, void *cuda_stream);

/* In-place GENP of C (Sec. 1.1; blocked form of block Gaussian elimination,
 * Thm. 2.2): right-looking with block size nb (0 = library default):
 * factor the nb x nb diagonal block, solve for the block row of U and the
 * block column of L, update the trailing Schur complement
 * A22 <- A22 - L21 U12, repeat.  On completion the strict lower triangle of
 * C holds L (unit diagonal implied) and the upper triangle holds U.
 *  C      n x n, ld ldc, double for FP64 and BF16_SLICED, float otherwise (caller-owned;
 *         the handle refers to it until destroyed or refactored).
 *  prec   GENP_FP64, GENP_FP32, GENP_BF16, GENP_BF16X3, GENP_FP8_E4M3 or
 *         GENP_BF16_SLICED (see genp_prec).
 *  nb     1 .. 128; 0 picks 128 for the tensor-core arithmetics (BF16,
 *         BF16X3, FP8_E4M3, BF16_SLICED) and 64 otherwise.
 *  out    receives a new factors handle (status word and workspace).
 * A zero or non-finite pivot does not stop the elimination; its step is
 * recorded (genp_info.breakdown_step, status GENP_ERR_BREAKDOWN) and the
 * factors are then meaningless.  No pivot threshold is applied. */
GENP_API genp_status genp_factor(void *C, int64_t n, int64_t ldc, genp_prec prec, int64_t nb, void *cuda_stream,
                        genp_factors **out);

/* Block Gaussian elimination of C with explicit inverses of the pivot
 * blocks (Sec. 2; Theorem 2.2 bounds the norms of the pivot blocks of block
 * Gaussian elimination and of their inverses for a strongly well
 * conditioned matrix, as it bounds GENP's pivots).  C is cut into nb x nb
 * diagonal blocks; at step k the leading block P_k of the current Schur
 * complement is inverted explicitly (Gauss-Jordan elimination without
 * pivoting), the block column below it becomes L_ik = S_ik P_k^{-1}, the
 * block row is kept (U_kj = S_kj), and the trailing matrix is updated,
 * S_ij <- S_ij - L_ik S_kj.  So C = L_B U_B with L_B block unit lower
 * (identity diagonal blocks) and U_B block upper with P_k on its diagonal.
 *  C      n x n FP64, ld ldc, in place (caller-owned; the handle refers to
 *         it): L_B below the block diagonal, U_B on and above it.  The
 *         inverses P_k^{-1} are kept in the handle.
 *  nb     64 (0 picks 64); other orders return GENP_ERR_UNSUPPORTED.
 *  out    a factors handle of precision GENP_FP64 that genp_solve,
 *         genp_refine (both methods), genp_adjoint, genp_refactor and
 *         genp_info_fetch accept like genp_factor's: the solves apply
 *         P_k^{-1} at each diagonal block.  genp_info's pivots are those met
 *         inside the Gauss-Jordan inversions (GENP's pivots of C), growth is
 *         max|U_B| / max|C|, and a zero or non-finite pivot is reported as a
 *         breakdown at its global step.
 * Errors: GENP_ERR_ARG, GENP_ERR_UNSUPPORTED, GENP_ERR_NOMEM, GENP_ERR_CUDA. */
GENP_API genp_status genp_block_factor(double *C, int64_t n, int64_t ldc, int64_t nb, void *cuda_stream,
                                       genp_factors **out);

/* Factors a new matrix of the same order and precision into an existing
 * handle, reusing its workspace (no allocation). */
GENP_API genp_status genp_refactor(genp_factors *F, void *C, int64_t ldc, void *cuda_stream);

/* Frees F (cudaFree waits for work still using it). NULL is ignored. */
GENP_API void genp_factors_destroy(genp_factors *F);

/* X = G U^{-1} L^{-1} B (Sec. 1.1: solve L U y = b, return x = G y).
 *  B, X   n x nrhs double, ld ldb / ldx; X may alias B only if ldx == ldb.
 *  The triangular solves run in the factor's precision, x = G y in FP64. */
GENP_API genp_status genp_solve(const genp_factors *F, const genp_multiplier *G, const double *B, int64_t ldb,
                       int64_t nrhs, double *X, int64_t ldx, void *cuda_stream);

/* Iterative refinement in FP64 (Sec. 7.1; Table 7.1 shows one step):
 *   repeat  r = B - A X (FP64);  C d = r (factor precision);  X += G d (FP64)
 * with the normwise backward error of every column,
 *   eta = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf),
 * measured before the first step and after each one.  Stops when
 * max eta <= tol, when eta fails to halve, or after max_iter steps; the
 * stop is decided on the device (no host synchronization).
 *  A      the ORIGINAL n x n matrix in double (C = A G), ld lda.
 *  X      on entry the solution of genp_solve, on exit the refined one.
 *  method 0 = classic refinement: d = U^{-1} L^{-1} r.
 *         1 = GMRES-IR (Carson and Higham): C d = r is solved by FP64
 *             GMRES on the left-preconditioned system
 *             U^{-1} L^{-1} A G d = U^{-1} L^{-1} r, at most
 *             GENP_GMRES_RESTART Krylov vectors per step, to a relative
 *             residual of 1e-10; C v is applied as A (G v).  It converges
 *             when the factors are only a fair preconditioner (low-precision
 *             factors of a matrix with large element growth), where classic
 *             refinement stagnates.  Needs (GENP_GMRES_RESTART + 4) n nrhs
 *             doubles of workspace (allocated by the library on first use).
 *  nrhs   at most 16.
 * genp_info.bwd_err / refine_iters report the history; status
 * GENP_ERR_NOCONV if the final eta is above tol. */
GENP_API genp_status genp_refine(const double *A, int64_t lda, const genp_factors *F, const genp_multiplier *G,
                        const double *B, int64_t ldb, int64_t nrhs, double *X, int64_t ldx, double tol,
                        int max_iter, int method, void *cuda_stream);

/* Refinement as one CUDA graph.  genp_refine enqueues its whole budget of
 * steps (max_iter outer steps, for GMRES-IR each with GENP_GMRES_RESTART
 * Krylov steps) and the device skips what it no longer needs, so a call is
 * thousands of launches, most of them skipped; on the host that is several
 * microseconds per launch.  With graphs on (the default), genp_refine
 * records that sequence once per set of arguments (A, G, B, X, their leading
 * dimensions, nrhs, tol, max_iter, method, the factors' matrix and
 * workspace) on a private stream into a CUDA graph kept in the factors
 * handle (up to four such graphs, replaced round robin; replacing one waits
 * for the device), and each call then launches the graph on the caller's
 * stream.  A call on a stream that is being captured enqueues its launches
 * one by one into the caller's capture instead.  While a graph is being
 * recorded the launch profile (genp_profile_*) leaves its launches out.
 *  enable  1 on, 0 off, -1 only queries.  Returns the previous setting. */
GENP_API int genp_refine_graphs(int enable);

/* Adjoint of X = A^{-1} B through the factors of C = A G: with gX = dl/dX,
 *   Lambda = A^{-T} gX = L^{-T} U^{-T} G^T gX,   dA = -Lambda X^T,   dB = Lambda.
 * (A^{-1} = G U^{-1} L^{-1}; the result does not depend on G in exact
 * arithmetic.)
 *  gX, X  n x nrhs double; dB n x nrhs double (may be NULL).
 *  dA     n x n, ld ldda, double for FP64 factors, float otherwise (may be NULL). */
GENP_API genp_status genp_adjoint(const genp_factors *F, const genp_multiplier *G, const double *gX, int64_t ldg,
                         const double *X, int64_t ldx, int64_t nrhs, void *dA, int64_t ldda, double *dB,
                         int64_t lddb, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Batched solves: many independent small systems (1 <= n_i <= 1024) in one
 * persistent launch.  Each system gets its own multiplier (stream id = its
 * index i, drawn in single precision: GENP_FP32 grid), its own FP32
 * factorization C_i = A_i G_i = L_i U_i and FP64 refinement; a work queue
 * hands the systems, largest first, to the CTAs.  The refinement is
 * GMRES-IR: r = b - A x in FP64, an FP32 GMRES on U^{-1} L^{-1} C_i d =
 * U^{-1} L^{-1} r (at most 16 Krylov steps, relative tolerance 1e-3; the
 * preconditioner applied through explicit FP32 inverses of L and U, or by
 * substitution once that stalls; a step that raises the backward error is
 * undone), then
 * x += G_i d in FP64 (Carson & Higham 2018), until the backward error is
 * <= tol, fails to halve on two outer steps in a row, or after max_iter
 * outer steps; FP32 elimination without
 * pivoting loses u32 times the element growth, which classic refinement
 * alone does not recover for Gaussian systems of order a few hundred.
 * The plan owns every workspace, so genp_batched_run allocates and
 * synchronizes nothing and can be captured in a CUDA graph.
 * Pools (caller-owned device memory) hold the systems back to back in the
 * caller's order: A_i (n_i x n_i, row-major, ld n_i) at mat_offsets[i],
 * B_i / X_i (n_i x nrhs, ld nrhs) at vec_offsets[i] (genp_batched_layout).
 * ---------------------------------------------------------------------- */
typedef struct genp_batched_plan genp_batched_plan;

/* count      number of systems (>= 1); n: host array of their orders.
 * nrhs       right-hand sides per system (1..16).
 * kind       GENP_MULT_GAUSSIAN (dense N(0, 1/n_i)) or GENP_MULT_CIRCULANT (N(0,1) first column).
 * a_prec     storage of the A pool: GENP_FP64 or GENP_FP32.
 * max_iter   outer refinement steps (0..32; 0 = no refinement), tol their
 *            target backward error.
 * flags      GENP_BATCH_AUTOTUNE: time the candidate CTA GEMM tiles (64 and
 *            128) of each size class once on this GPU (synchronizes; the
 *            choice is kept per process and, if GENP_AUTOTUNE_CACHE names a
 *            file, there).
 *            GENP_BATCH_FP64_ESCALATION: a second launch after each run
 *            factors every system whose refinement did not reach tol again
 *            in double-float arithmetic (about 48 bits) and refines it with
 *            those factors (the plan then holds 8.1 MiB of scratch per
 *            persistent CTA of that launch).
 * Errors: GENP_ERR_ARG, GENP_ERR_NOMEM, GENP_ERR_CUDA. */
#define GENP_BATCH_AUTOTUNE 1
#define GENP_BATCH_FP64_ESCALATION 2
GENP_API genp_status genp_batched_plan_create(int64_t count, const int64_t *n, int64_t nrhs, genp_mult_kind kind,
                                              genp_prec a_prec, int max_iter, double tol, int flags,
                                              void *cuda_stream, genp_batched_plan **out);

/* Host arrays of count+1 entries: element offsets of every system in the A
 * pool and in the B / X pools (the last entry is the pool size). */
GENP_API genp_status genp_batched_layout(const genp_batched_plan *P, int64_t *mat_offsets, int64_t *vec_offsets);

/* CTA GEMM tile (64 or 128) the plan uses for systems of order n (after
 * autotuning); the factorization block is 32. */
GENP_API int genp_batched_block_size(const genp_batched_plan *P, int64_t n);

/* Draws every system's multiplier from `seed` (system i: stream id i) and
 * solves all systems: X_i = A_i^{-1} B_i by the method, refined in FP64.
 * A pool in a_prec; B and X pools double.  Keeps the factors for
 * genp_batched_adjoint. */
GENP_API genp_status genp_batched_run(genp_batched_plan *P, uint64_t seed, const void *A_pool, const double *B_pool,
                                      double *X_pool, void *cuda_stream);

/* Adjoint of the last run through its factors: Lambda_i = A_i^{-T} gX_i =
 * L_i^{-T} U_i^{-T} G_i^T gX_i, refined in FP64 against the A pool like the
 * forward solve (same max_iter and tol); dB_i = Lambda_i (double, may be
 * NULL); dA_i = -Lambda_i X_i^T (float, A-pool layout, may be NULL). */
GENP_API genp_status genp_batched_adjoint(genp_batched_plan *P, const void *A_pool, const double *gX_pool,
                                          const double *X_pool, float *dA_pool, double *dB_pool, void *cuda_stream);

/* Per-system results of the last run (host arrays of count entries, any may
 * be NULL): status (GENP_OK / GENP_ERR_BREAKDOWN / GENP_ERR_NOCONV), outer
 * refinement steps, backward error before and after refinement, growth
 * max|U| / max|C| of the FP32 factorization, its escalation level (0: the
 * inner solves used the explicit inverses of the factors throughout; 1: they
 * switched to substitution with L and U after a stall; 2: refactored in
 * double-float by the escalation launch), and the inner Krylov steps taken.
 * Synchronizes the stream. */
GENP_API genp_status genp_batched_status(const genp_batched_plan *P, int32_t *status, int32_t *iters, double *eta0,
                                         double *eta, double *growth, int32_t *escalated, int32_t *krylov,
                                         void *cuda_stream);

/* Copies the multipliers of the last run into caller pools: dense G_i
 * (float, A-pool layout) or circulant first columns g_i (float, sum n_i,
 * back to back in the caller's order). */
GENP_API genp_status genp_batched_multipliers(const genp_batched_plan *P, float *G_pool, float *g_pool,
                                              void *cuda_stream);

/* Phase profile of the batched kernel (diagnostics).  enable != 0 makes
 * every later run record, per persistent CTA, the SM cycles spent in each
 * phase of its last run; genp_batched_profile_read sums them over the CTAs
 * into cycles[7]: C = A G, factorization, inverses of the factors, first
 * solve and x = G y, FP64 residuals, inner GMRES, x += G d.  The read
 * synchronizes the stream. */
GENP_API genp_status genp_batched_profile(genp_batched_plan *P, int enable);
GENP_API genp_status genp_batched_profile_read(const genp_batched_plan *P, double *cycles, void *cuda_stream);

/* Frees the plan (cudaFree waits for work still using it). NULL is ignored. */
GENP_API void genp_batched_plan_destroy(genp_batched_plan *P);

/* Tensor-core building block of the BF16 path (tcgen05, FP32 accumulation):
 *   D = alpha * A * B^T + beta * Cin
 *  A      m x K BF16 (uint16 storage), row-major, ld lda (multiple of 8,
 *         16-byte aligned base).
 *  Bt     n x K BF16, row-major, ld ldb (same rules); i.e. B^T.
 *  Cin, D m x n FP32, ld ldci / ldd; Cin may be NULL when beta == 0 and may
 *         equal D (in-place update).
 * Errors: GENP_ERR_ARG (sizes, alignment), GENP_ERR_CUDA. */
GENP_API genp_status genp_gemm_bf16(int64_t m, int64_t n, int64_t K, float alpha, const void *A, int64_t lda,
                                    const void *Bt, int64_t ldb, float beta, const float *Cin, int64_t ldci,
                                    float *D, int64_t ldd, void *cuda_stream);

/* E4M3 operands with one power-of-two scale per 128 x 128 tile (the
 * operands of GENP_FP8_E4M3).  For the logical operand X (m x K):
 *   X = src (m x K, ld lds) when trans == 0, X = src^T (src K x m) otherwise.
 * Tile (ti, kt) covers rows 128 ti .. and columns 128 kt ..; its scale is
 * 2^e with e the least integer such that max |X_tile| <= 448 2^e (448: the
 * largest finite e4m3 value), clamped to [-126, 126]; e = 0 for a zero tile.
 *   dst[i ldq + k]               = e4m3 code of X[i][k] 2^-e, rounded to
 *                                  nearest, ties to even (the scaling is exact)
 *   scales[ti ceil(K/128) + kt]  = 2^e (float)
 * src device FP64 or FP32 (src_prec); dst device bytes, ldq >= K, a multiple
 * of 16, base 16-byte aligned; entries k >= K of a row are not written.
 * Errors: GENP_ERR_ARG, GENP_ERR_CUDA. */
GENP_API genp_status genp_quantize_e4m3(const void *src, int64_t lds, genp_prec src_prec, int64_t m, int64_t K,
                                        int trans, uint8_t *dst, int64_t ldq, float *scales, void *cuda_stream);

/* Tensor-core product of tile-scaled e4m3 operands (tcgen05 kind::f8f6f4,
 * FP32 accumulation of each run of 128-wide k-tiles with one scale product,
 * promoted into FP32 with that scale):
 *   D = alpha * sum_kt scale_a[tm][kt] scale_b[tn][kt] A_kt Bt_kt^T + beta * Cin
 *  A   m x K codes, ld lda; scale_a ceil(m/128) x ceil(K/128) floats.
 *  Bt  n x K codes (B transposed), ld ldb; scale_b ceil(n/128) x ceil(K/128).
 *  lda, ldb multiples of 16, bases 16-byte aligned; Cin, D as genp_gemm_bf16;
 *  K <= 262144.  Consecutive k-tiles with the same scale product accumulate
 *  together in FP32 on the tensor cores before the promotion.
 * Errors: GENP_ERR_ARG, GENP_ERR_CUDA. */
GENP_API genp_status genp_gemm_e4m3(int64_t m, int64_t n, int64_t K, float alpha, const uint8_t *A, int64_t lda,
                                    const float *scale_a, const uint8_t *Bt, int64_t ldb, const float *scale_b,
                                    float beta, const float *Cin, int64_t ldci, float *D, int64_t ldd,
                                    void *cuda_stream);

/* Randomized low-rank approximation (Sec. 5, Proto-Alg. 5.1, with an
 * orthonormal T as in the tests of Sec. 7.2):
 *   Stage 1  B = A^T G with an m x r sketch G: GENP_MULT_GAUSSIAN (iid
 *            N(0,1), Definition 3.2) or GENP_MULT_TOEPLITZ (Gaussian
 *            Toeplitz, the multipliers of Table 7.3), drawn from
 *            (seed, stream_id) on their own Philox tags;
 *   basis    B = Q R, Q n x r orthonormal, R upper triangular with a
 *            positive diagonal (so Q is unique, Fact 2.2), by shifted
 *            Cholesky QR in three passes (CholeskyQR3);
 *   Stage 3  A Q, so the rank-r approximation is A_hat = (A Q) Q^T.
 *  A      m x n FP64 (ld lda), device.
 *  r      1 <= r <= min(n, 128).
 *  G      NULL or m x r (ld ldg): receives the sketch.
 *  Q      n x r (ld ldq), required.  R: NULL or r x r (ld ldr), R = Q^T B.
 *  AQ     NULL or m x r (ld ldaq).
 *  dev_status  NULL or a device int: 0, or k + 1 if a Cholesky pass met a
 *         non-positive pivot at step k (B numerically rank deficient
 *         beyond what the shift covers); written before the call's work
 *         completes on the stream.
 * Allocates its workspace with cudaMallocAsync on the stream.
 * Errors: GENP_ERR_ARG (sizes, kind), GENP_ERR_NOMEM, GENP_ERR_CUDA. */
GENP_API genp_status genp_lowrank(int64_t m, int64_t n, const double *A, int64_t lda, int64_t r, genp_mult_kind kind,
                                  uint64_t seed, uint64_t stream_id, double *G, int64_t ldg, double *Q, int64_t ldq,
                                  double *R, int64_t ldr, double *AQ, int64_t ldaq, int *dev_status,
                                  void *cuda_stream);

/* Numerical rank without pivoting or orthogonalization (App. B,
 * Proto-Alg. B.1).  With the m x r_hi Gaussian sketch G drawn once from
 * (seed, stream_id) (the tag of genp_lowrank's Gaussian sketch) and G_r its
 * first r columns, B' = A^T G_r is full rank and well conditioned exactly
 * when r does not exceed the numerical rank (Thm. 5.1).  As printed, the
 * algorithm's update (a passing test lowers the top of the range) would
 * settle on the smallest passing r; this entry point searches for the
 * largest: r = ceil((r_lo + r_hi) / 2) (Remark B.4), pass -> r_lo = r,
 * fail -> r_hi = r - 1, until r_lo = r_hi.  COND (Remark B.2): Cholesky of
 * B'^T B' without pivoting, 40 power steps for its largest eigenvalue and
 * 40 inverse-iteration steps for its smallest; pass when the resulting
 * kappa_2(B') <= cond_max.
 *  A        m x n FP64 (ld lda), device.   0 <= r_lo <= r_hi <= min(n, 128).
 *  rank     host: the numerical rank found.
 *  B        NULL or n x r_hi (ld ldb): receives A^T G_rank (rank columns).
 * Synchronizes the stream once per candidate r (the search branches on the
 * device's answer).  Allocates its workspace with cudaMallocAsync.
 * Errors: GENP_ERR_ARG, GENP_ERR_NOMEM, GENP_ERR_CUDA. */
GENP_API genp_status genp_numerical_rank(int64_t m, int64_t n, const double *A, int64_t lda, int64_t r_lo,
                                         int64_t r_hi, double cond_max, uint64_t seed, uint64_t stream_id,
                                         int64_t *rank, double *B, int64_t ldb, void *cuda_stream);

/* Tensor-core building block of the BF16_SLICED path:
 *   D = alpha * A * B + beta * D      (all FP64, row-major)
 * with A * B formed on the BF16 tensor cores from exact 7-bit digit slices
 * (see GENP_BF16_SLICED), in K chunks of at most 512 summed in
 * double-float, and one rounding to FP64 at the end.  Per entry and chunk
 * the error is about 2^-(7 digits - 1) * 4 * K_c * max_k|a_ik| * max_k|b_kj|
 * at worst (far less for sums with mixed signs); products of integers with
 * |a|, |b| <= 127 are exact for K <= 2^20.  digits: 3 to 7, or 0 (the
 * setting of genp_sliced_digits).
 *  A      m x K, ld lda;  B  K x n, ld ldb;  D  m x n, ld ldd.
 *  Allocates its workspace with cudaMallocAsync on the stream.
 * Errors: GENP_ERR_ARG (sizes), GENP_ERR_NOMEM, GENP_ERR_CUDA. */
GENP_API genp_status genp_gemm_sliced(int64_t m, int64_t n, int64_t K, double alpha, const double *A, int64_t lda,
                                      const double *B, int64_t ldb, double beta, double *D, int64_t ldd, int digits,
                                      void *cuda_stream);

/* Digits per operand of the BF16_SLICED path: 5 (15 digit products per
 * multiply-add, about 32 correct bits on Gaussian data), 6 (21, about 39) or
 * 7 (28, about 46; the default).  digits == 0 returns the current setting;
 * otherwise sets it for every later genp_factor / genp_precondition /
 * genp_gemm_sliced call of the process and returns the previous one, or -1
 * if digits is not supported.  Not synchronized with concurrent calls. */
GENP_API int genp_sliced_digits(int digits);

/* Digits per operand of the sliced product C = A G that genp_precondition
 * forms for a Gaussian multiplier when c_prec is GENP_BF16_SLICED: 3 to 7
 * (6, 10, 15, 21 or 28 digit products per multiply-add; about 19, 26, 33,
 * 40 or 47 correct bits on Gaussian data); default 7.  The refinement's
 * residual b - A x and its update x += G d use A and G in FP64 (Thm. 4.1
 * allows the product to be perturbed), so the product only has to be as
 * accurate as the factors it feeds: with GMRES-IR (genp_refine method 1),
 * which needs the factors only as a preconditioner, 4 or 5 digits reach
 * the same final backward error.  Classic refinement contracts only while
 * kappa(A G) times the product's relative error stays below one, so it
 * wants the default.  digits == 0 returns the current setting; otherwise
 * sets it for later genp_precondition calls of the process and returns the
 * previous one, or -1 if digits is not supported.  Not synchronized with
 * concurrent calls. */
GENP_API int genp_sliced_precondition_digits(int digits);

/* Digits of the sliced grid (value_grid GENP_BF16_SLICED) of the dense
 * Gaussian multipliers created afterwards: 1 (the default; multiples of
 * 2^(E - 6)) or 2 (multiples of 2^(E - 13)); circulant and Toeplitz
 * multipliers keep two.  Thm. 4.1's perturbed Gaussian G = G' + U covers
 * either grid, and GENP of A G with the coarser one leaves the pivots'
 * growth and the unrefined backward error at the two-digit grid's level on
 * Gaussian test matrices; with one digit the sliced C = A G forms nd digit
 * products per multiply-add (nd = genp_sliced_precondition_digits) instead
 * of 2 nd - 1.  A multiplier keeps the grid it was created with (redraws
 * included).  digits == 0 returns the current setting; 1 or 2 sets it and
 * returns the previous one; anything else returns -1.  Not synchronized
 * with concurrent calls. */
GENP_API int genp_sliced_multiplier_digits(int digits);

/* Measurement hook: while enabled, every launch of the sliced and the e4m3
 * tensor-core kernels is bracketed by two CUDA events on its stream.
 * genp_profile_read synchronizes on them and returns the summed kernel time
 * (ms), the flops (sliced: the digit products' BF16 flops, 2 m n Kpad x
 * digit pairs per launch; e4m3: 2 m n K) and the launch count since the last
 * read or enable, then restarts the count.  genp_profile_launches returns
 * the same launches one by one, in launch order (the first min(cap, count)
 * into ms[] and flops[], either may be NULL), and the count, without
 * restarting it.  Enabling costs two event records per launch; it is off by
 * default. */
GENP_API genp_status genp_profile_enable(int on);
GENP_API genp_status genp_profile_read(double *ms, double *flops, int *launches);
GENP_API genp_status genp_profile_launches(double *ms, double *flops, int cap, int *launches);
/* The same hook by kernel class, each launch counted with its algorithmic
 * work:
 *  GENP_PROF_TENSOR (0): the tensor-core launches above; work = the
 *      product's own flops, 2 m n K per launch (for the sliced product the
 *      FP64-class product it forms, not its digit products).
 *  GENP_PROF_TRSV (1): the streaming triangular solves (Sec. 1.1, L U y = b);
 *      work = bytes of the triangular factor read, n^2 / 2 x 8 B per pass
 *      and RHS chunk (FP64 or double-float factors; 4 B per entry for FP32).
 *  GENP_PROF_GEMV (2): matrix-vector products (x = G y, r = b - A x, the
 *      Krylov products A (G v)); work = bytes of the matrix read, m k x
 *      element size per launch.
 *  GENP_PROF_FACTOR_AUX (3): the factorization's kernels off the tensor
 *      cores (diagonal blocks, block row and column, the pivot-block
 *      inverses of block GE); work = flops (nb^3 2/3 per diagonal block,
 *      nb^2 w per block row or column of width w).
 *  GENP_PROF_OUTER (4): the adjoint's dA = -Lambda X^T; work = bytes of dA
 *      written.
 *  GENP_PROF_PRECOND (5): C = A G for the circulant (FFT) and sparse
 *      (signed gather) multipliers in FP64; work = 16 n^2 bytes (A read, C
 *      written).
 * Returns the summed time (ms), work and launch count of class `cls` since
 * the last genp_profile_enable, synchronizing on their events; does not
 * restart the count.  Launches that returned at once because the
 * device-steered refinement had already stopped (classes 1 and 2) count
 * their time and launch but not their work.  GENP_ERR_ARG for another
 * class. */
#define GENP_PROF_TENSOR 0
#define GENP_PROF_TRSV 1
#define GENP_PROF_GEMV 2
#define GENP_PROF_FACTOR_AUX 3
#define GENP_PROF_OUTER 4
#define GENP_PROF_PRECOND 5
GENP_API genp_status genp_profile_class(int cls, double *ms, double *work, int *launches);

/* Synchronizes the device and reports whether any kernel of this library
 * that waits on the device (the tensor-core pipelines, the persistent
 * triangular solves) gave up a bounded wait (GENP_ERR_TIMEOUT) since the
 * last clear; `clear` != 0 resets the flags.  GENP_OK otherwise. */
GENP_API genp_status genp_device_check(int clear);

/* Allocation-free draw of the SPARSE_PM1 multiplier.  The paper has no
 * counterpart: this serves callers that cannot call cudaMalloc, such as code
 * whose device memory all belongs to another allocator (a framework pool that
 * has already reserved it, an application that maps its memory once at
 * start-up) or a latency-critical loop that must not pay the device-wide
 * synchronization cudaMalloc / cudaFree can cause.
 * Writes the same multiplier as genp_make_multiplier(GENP_MULT_SPARSE_PM1, n,
 * seed, stream_id, ...) into caller-owned device buffers, each nnz_per_col*n:
 *  rows[t*n + j]      row of the t-th entry of column j (int32)
 *  signs[t*n + j]     its sign (int8, +1 or -1)
 *  inv_rows[t*n + i]  column whose t-th entry sits in row i (int32)
 *  inv_signs[t*n + i] that entry's sign (int8)
 * Its only scratch (the Fisher-Yates swap draws) is a file-scope device array
 * of GENP_NOALLOC_MAX_ENTRIES int32 (4 MiB) that every GPU loading the
 * library holds until the process exits; n * nnz_per_col above that limit
 * returns GENP_ERR_ARG with nothing enqueued.  Nothing in the array needs
 * clearing between calls (each call writes every entry it reads), but all
 * calls on one GPU share it: calls whose work overlaps on the same GPU (two
 * streams, or two host threads enqueueing at once) race and corrupt each
 * other's result.  Serialize them on one stream.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and keeps it for the
 * life of the process; make that first call before any stream capture.
 * cudaDeviceReset unloads the array with the rest of the module, so the
 * kept address is stale afterwards: do not call this entry point on a
 * device after resetting it in the same process.  No cudaMalloc, cudaFree or allocating library
 * routine is called.  Errors: GENP_ERR_ARG, GENP_ERR_CUDA. */
#define GENP_NOALLOC_MAX_ENTRIES (1 << 20)
GENP_API genp_status genp_make_sparse_noalloc(int64_t n, int nnz_per_col, uint64_t seed, uint64_t stream_id,
                                              int32_t *rows, int8_t *signs, int32_t *inv_rows, int8_t *inv_signs,
                                              void *cuda_stream);

/* Number of kernels this library has launched in the process so far
 * (diagnostics: lets a caller count the launches of a timed region).  The
 * steps of a recorded refinement graph that a converged refinement skips
 * launch nothing and are not counted; the kernels of the steps that ran are
 * added on the device, into pinned host memory, so the count is complete
 * once the caller has synchronized the stream.  That pinned word belongs to
 * the device's context: after cudaDeviceReset in the process, do not call
 * this function again. */
GENP_API uint64_t genp_launch_count(void);

/* Copies the device status of F to *out after synchronizing cuda_stream. */
GENP_API genp_status genp_info_fetch(const genp_factors *F, genp_info *out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* GENP_H */
