// api.cu -- the extern "C" entry points declared in include/genp.h.
//
// Every entry point checks its arguments on the host (returning
// GENP_ERR_ARG with nothing enqueued), then only enqueues kernels on the
// caller's stream.  Handles own their device storage; caller buffers are
// never freed or retained (except the C buffer a factors handle refers to).
#include "genp_internal.cuh"

#include <math.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <new>
#include <vector>

using namespace genp;

namespace {

std::atomic<uint64_t> g_launches{0};
// kernels of the conditional bodies that recorded refinement graphs ran: the
// IF nodes' condition kernels add them up in pinned host memory (one thread
// each, ordered by the graph), so the count needs no copy or synchronization
unsigned long long *g_body_launches = nullptr;       // host view
unsigned long long *g_body_launches_dev = nullptr;   // device view
std::mutex g_body_launches_mu;

cudaStream_t S(void *p) { return static_cast<cudaStream_t>(p); }

template <typename T>
genp_status dalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) return GENP_OK;
    if (cudaMalloc((void **)p, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return GENP_ERR_NOMEM;
    }
    return GENP_OK;
}

#define TRY(expr)                                        \
    do {                                                 \
        genp_status st_ = (expr);                        \
        if (st_ != GENP_OK) return st_;                  \
    } while (0)
#define CU(expr)                                         \
    do {                                                 \
        if ((expr) != cudaSuccess) {                     \
            cudaGetLastError();                          \
            return GENP_ERR_CUDA;                        \
        }                                                \
    } while (0)

void free_multiplier(genp_multiplier *G) {
    cudaFree(G->dense);
    cudaFree(G->dense_f32);
    cudaFree(G->dense_bf16);
    cudaFree(G->g);
    cudaFree(G->spec);
    cudaFree(G->spec_f32);
    cudaFree(G->twid);
    cudaFree(G->twid_f32);
    cudaFree(G->rows);
    cudaFree(G->signs);
    cudaFree(G->inv_rows);
    cudaFree(G->inv_signs);
    cudaFree(G->draws);
    cudaFree(G->attempt);
    delete G;
}

// Enqueues the draw of G's entries from (seed, stream_id) into its storage.
cudaError_t draw_multiplier(genp_multiplier *G, uint64_t seed, uint64_t stream_id, cudaStream_t s) {
    switch (G->kind) {
        case GENP_MULT_GAUSSIAN:
            return launch_make_dense(G->dense, G->n, seed, stream_id, G->scale, G->grid, G->dense_f32, G->dense_bf16,
                                     s, G->grid_digits);
        case GENP_MULT_CIRCULANT: {
            cudaError_t e = G->pm1        ? launch_make_circulant_pm1(G->g, G->n, seed, stream_id, G->attempt, s)
                            : G->toeplitz ? launch_make_toeplitz(G->g, G->n, seed, stream_id, G->scale, G->grid, s)
                                          : launch_make_circulant(G->g, G->n, seed, stream_id, G->scale, G->grid, s);
            return e == cudaSuccess ? circ_prepare(G, s) : e;
        }
        case GENP_MULT_HOUSEHOLDER_PM1: return launch_make_householder(G->g, G->n, seed, stream_id, s);
        case GENP_MULT_IDENTITY: return cudaSuccess;
        case GENP_MULT_SPARSE_PM1:
            return launch_make_sparse(G->rows, G->signs, G->inv_rows, G->inv_signs, G->draws, G->n, G->nnz, seed,
                                      stream_id, s);
    }
    return cudaErrorInvalidValue;
}

bool factor_prec_ok(genp_prec p) {
    return p == GENP_FP64 || p == GENP_FP32 || p == GENP_BF16 || p == GENP_BF16X3 || p == GENP_BF16_SLICED ||
           p == GENP_FP8_E4M3;
}
// FP32 master copy, Schur products on the tensor cores (BF16 or e4m3 operands)
bool tc_prec(genp_prec p) { return p == GENP_BF16 || p == GENP_BF16X3 || p == GENP_FP8_E4M3; }

// Grows the factors workspace to at least `bytes` (synchronizes the stream
// only when it actually has to grow).
genp_status ensure_work(genp_factors *F, size_t bytes, cudaStream_t s) {
    if (F->work_bytes >= bytes) return GENP_OK;
    if (F->work) {
        CU(cudaStreamSynchronize(s));
        cudaFree(F->work);
        F->work = nullptr;
        F->work_bytes = 0;
    }
    if (cudaMalloc(&F->work, bytes) != cudaSuccess) {
        cudaGetLastError();
        F->work = nullptr;
        return GENP_ERR_NOMEM;
    }
    F->work_bytes = bytes;
    return GENP_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Stream-ordered workspaces (cudaMallocAsync) come from the device's default
// memory pool; by default the pool hands freed memory back to the driver at
// every synchronization, and the next call maps it again.  On first use per
// device the library keeps the pool's memory cached instead.
void keep_pool_cached() {
    static std::atomic<uint64_t> done{0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return;
    }
    const uint64_t bit = 1ull << dev;
    if (done.load(std::memory_order_relaxed) & bit) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    done.fetch_or(bit, std::memory_order_relaxed);
}

}  // namespace

namespace genp {

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(uint64_t count) { g_launches.fetch_add(count, std::memory_order_relaxed); }

// X[r][c] += Y[r][c] (the identity multiplier's x += G d)
__global__ void k_add_into(const double *Y, int64_t ldy, double *X, int64_t ldx, int64_t n, int64_t nr,
                           const int *skip) {
    if (skip && *skip) return;
    for (int64_t r = blockIdx.y; r < n; r += gridDim.y)
        for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nr; c += (int64_t)gridDim.x * blockDim.x)
            X[r * ldx + c] += Y[r * ldy + c];
}
// G = I into a dense buffer
__global__ void k_eye(double *G, int64_t n, int64_t ldg) {
    for (int64_t r = blockIdx.y; r < n; r += gridDim.y)
        for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
            G[r * ldg + c] = r == c ? 1.0 : 0.0;
}

cudaError_t add_into(const double *Y, int64_t ldy, double *X, int64_t ldx, int64_t n, int64_t nr, const int *skip,
                     cudaStream_t s) {
    if (n <= 0 || nr <= 0) return cudaSuccess;
    note_launch();
    k_add_into<<<dim3((unsigned)cdiv(nr, 32), (unsigned)(n < 65535 ? n : 65535)), 32, 0, s>>>(Y, ldy, X, ldx, n, nr,
                                                                                           skip);
    return cudaGetLastError();
}

cudaError_t apply_multiplier(const genp_multiplier *G, bool trans, const double *Y, int64_t ldy, double *X,
                             int64_t ldx, int64_t nrhs, bool accumulate, const int *skip, cudaStream_t s) {
    switch (G->kind) {
        case GENP_MULT_GAUSSIAN:
            return gemm<double>(G->n, nrhs, G->n, 1.0, G->dense, G->n, trans, Y, ldy, accumulate ? 1.0 : 0.0, X, ldx,
                                X, ldx, skip, s);
        case GENP_MULT_CIRCULANT:
            if (circ_fft_supported(G->cn))
                return circ_apply_cols(G, trans, Y, ldy, X, ldx, nrhs, accumulate, skip, s);
            return circ_apply_direct(G->g, G->cn, G->n, trans, Y, ldy, X, ldx, nrhs, accumulate, skip, s);
        case GENP_MULT_HOUSEHOLDER_PM1:   // symmetric: G^T = G
            return house_apply(G, Y, ldy, X, ldx, nrhs, accumulate, skip, s);
        case GENP_MULT_SPARSE_PM1:
            return sparse_apply(G, trans, Y, ldy, X, ldx, nrhs, accumulate, skip, s);
        case GENP_MULT_IDENTITY:
            if (!accumulate) return convert_matrix<double, double>(Y, ldy, X, ldx, G->n, nrhs, skip, s);
            note_launch();
            k_add_into<<<dim3((unsigned)cdiv(nrhs, 32), (unsigned)(G->n < 65535 ? G->n : 65535)), 32, 0, s>>>(
                Y, ldy, X, ldx, G->n, nrhs, skip);
            return cudaGetLastError();
        default: break;
    }
    return cudaErrorInvalidValue;
}

}  // namespace genp

namespace genp {

// The recording state of a refinement graph's conditional bodies (nesting:
// the graph, a residual check or correction, a Krylov step).
struct CondRec {
    static constexpr int kMaxBodies = (GENP_MAX_REFINE + 1) * (GENP_GMRES_RESTART + 2);
    cudaStream_t chain[3] = {};          // the graph's stream, then the nested bodies'
    int depth = 0;
    int idx[3] = {};
    uint64_t start[3] = {}, nested[3] = {};   // launch count at a body's start, its nested bodies' kernels
    std::vector<int> counts;             // kernels of each body, not counting the bodies nested in it
    int *dev_counts = nullptr;           // their device copy, read by the condition kernels
};

namespace {
// Sets the condition of the IF node that follows: run the body while *done
// is 0, and count its kernels.
__global__ void k_cond_set(cudaGraphConditionalHandle h, const int *done, const int *counts, int idx,
                           unsigned long long *launched) {
    const bool go = *done == 0;
    cudaGraphSetConditional(h, go ? 1u : 0u);
    if (go) {
        volatile unsigned long long *p = launched;
        *p = *p + (unsigned long long)counts[idx];
    }
}
}  // namespace

cudaError_t cond_begin(CondRec *c, cudaStream_t &s, const int *done) {
    if (!c) return cudaSuccess;
    if (c->depth >= 2 || (int)c->counts.size() >= CondRec::kMaxBodies) return cudaErrorInvalidValue;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusActive || !g) return cudaErrorStreamCaptureInvalidated;
    cudaGraphConditionalHandle h;
    e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return e;
    const int idx = (int)c->counts.size();
    c->counts.push_back(0);
    note_launch();
    k_cond_set<<<1, 1, 0, s>>>(h, done, c->dev_counts, idx, g_body_launches_dev);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd);
    if (e != cudaSuccess) return e;
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &p);
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) return e;
    cudaStream_t child = c->chain[c->depth + 1];
    e = cudaStreamBeginCaptureToGraph(child, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    ++c->depth;
    c->idx[c->depth] = idx;
    c->start[c->depth] = g_launches.load(std::memory_order_relaxed);
    c->nested[c->depth] = 0;
    s = child;
    return cudaSuccess;
}

cudaError_t cond_end(CondRec *c, cudaStream_t &s) {
    if (!c) return cudaSuccess;
    const int d = c->depth;
    if (d <= 0 || s != c->chain[d]) return cudaErrorInvalidValue;
    cudaGraph_t body = nullptr;   // owned by its IF node
    const cudaError_t e = cudaStreamEndCapture(s, &body);
    const uint64_t total = g_launches.load(std::memory_order_relaxed) - c->start[d];
    c->counts[c->idx[d]] = (int)(total - c->nested[d]);
    c->nested[d - 1] += total;
    c->depth = d - 1;
    s = c->chain[d - 1];
    return e;
}

}  // namespace genp

extern "C" {

const char *genp_version(void) { return "genp 0.1 sm_103a"; }

const char *genp_status_string(genp_status s) {
    switch (s) {
        case GENP_OK: return "GENP_OK";
        case GENP_ERR_ARG: return "GENP_ERR_ARG: invalid argument";
        case GENP_ERR_BREAKDOWN: return "GENP_ERR_BREAKDOWN: zero or non-finite pivot";
        case GENP_ERR_NOCONV: return "GENP_ERR_NOCONV: refinement did not reach the tolerance";
        case GENP_ERR_CUDA: return "GENP_ERR_CUDA: CUDA runtime error";
        case GENP_ERR_TIMEOUT: return "GENP_ERR_TIMEOUT: bounded device wait gave up";
        case GENP_ERR_NOMEM: return "GENP_ERR_NOMEM: device allocation failed";
        case GENP_ERR_UNSUPPORTED: return "GENP_ERR_UNSUPPORTED: combination not offered by the library";
    }
    return "unknown genp status";
}

genp_status genp_make_multiplier(genp_mult_kind kind, int64_t n, uint64_t seed, uint64_t stream_id, double scale,
                                 int nnz_per_col, genp_prec value_grid, void *cuda_stream, genp_multiplier **out) {
    if (!out) return GENP_ERR_ARG;
    *out = nullptr;
    if (n < 1 || n > 2147483647LL) return GENP_ERR_ARG;
    if (kind != GENP_MULT_GAUSSIAN && kind != GENP_MULT_CIRCULANT && kind != GENP_MULT_SPARSE_PM1 &&
        kind != GENP_MULT_CIRCULANT_PM1 && kind != GENP_MULT_IDENTITY && kind != GENP_MULT_TOEPLITZ &&
        kind != GENP_MULT_HOUSEHOLDER_PM1)
        return GENP_ERR_ARG;
    const bool pm1 = kind == GENP_MULT_CIRCULANT_PM1;
    if (pm1) {   // stored and applied as a circulant with a +-1 first column
        kind = GENP_MULT_CIRCULANT;
        scale = 1.0;
    }
    const bool toeplitz = kind == GENP_MULT_TOEPLITZ;
    if (toeplitz) {   // the leading block of a circulant of order 2n
        if (n > 1073741823LL) return GENP_ERR_ARG;
        kind = GENP_MULT_CIRCULANT;
    }
    if (kind == GENP_MULT_IDENTITY || kind == GENP_MULT_HOUSEHOLDER_PM1) {
        scale = 1.0;
        value_grid = GENP_FP64;
    }
    if (kind != GENP_MULT_SPARSE_PM1 && !(scale > 0.0 && isfinite(scale))) return GENP_ERR_ARG;
    if (kind == GENP_MULT_SPARSE_PM1 && (nnz_per_col < 1 || nnz_per_col > 16)) return GENP_ERR_ARG;
    if (value_grid != GENP_FP64 && value_grid != GENP_FP32 && value_grid != GENP_BF16 &&
        value_grid != GENP_FP8_E4M3 && value_grid != GENP_BF16_SLICED)
        return GENP_ERR_ARG;
    cudaStream_t s = S(cuda_stream);
    genp_multiplier *G = new (std::nothrow) genp_multiplier();
    if (!G) return GENP_ERR_NOMEM;
    G->kind = kind;
    G->n = n;
    G->nnz = kind == GENP_MULT_SPARSE_PM1 ? nnz_per_col : 0;
    G->grid = kind == GENP_MULT_SPARSE_PM1 ? GENP_FP64 : value_grid;
    G->grid_digits = (kind == GENP_MULT_GAUSSIAN && value_grid == GENP_BF16_SLICED) ? sliced_mult_digits() : 2;
    G->scale = kind == GENP_MULT_SPARSE_PM1 ? 1.0 : scale;
    G->pm1 = pm1;
    G->toeplitz = toeplitz;
    G->cn = toeplitz ? 2 * n : n;
    G->last_stream = s;
    genp_status st = GENP_OK;
    cudaError_t ce = cudaSuccess;
    if (kind == GENP_MULT_GAUSSIAN) {
        st = dalloc(&G->dense, (size_t)n * n);
        if (st == GENP_OK && value_grid != GENP_FP64 && value_grid != GENP_BF16_SLICED)
            st = dalloc(&G->dense_f32, (size_t)n * n);
        if (st == GENP_OK && value_grid == GENP_BF16) st = dalloc(&G->dense_bf16, (size_t)n * round8(n));
    } else if (kind == GENP_MULT_IDENTITY) {
        // nothing to store
    } else if (kind == GENP_MULT_HOUSEHOLDER_PM1) {
        st = dalloc(&G->g, (size_t)n);
    } else if (kind == GENP_MULT_CIRCULANT) {
        const int64_t cn = G->cn;
        st = dalloc(&G->g, (size_t)cn);
        if (st == GENP_OK && pm1) st = dalloc(&G->attempt, 1);
        if (st == GENP_OK && circ_fft_supported(cn)) {
            st = dalloc(&G->spec, (size_t)cn);
            if (st == GENP_OK) st = dalloc(&G->spec_f32, (size_t)cn);
            if (st == GENP_OK) st = dalloc(&G->twid, (size_t)(cn / 2));
            if (st == GENP_OK) st = dalloc(&G->twid_f32, (size_t)(cn / 2));
        }
    } else {
        const size_t cnt = (size_t)n * nnz_per_col;
        st = dalloc(&G->rows, cnt);
        if (st == GENP_OK) st = dalloc(&G->signs, cnt);
        if (st == GENP_OK) st = dalloc(&G->inv_rows, cnt);
        if (st == GENP_OK) st = dalloc(&G->inv_signs, cnt);
        if (st == GENP_OK) st = dalloc(&G->draws, cnt);
    }
    if (st == GENP_OK) ce = draw_multiplier(G, seed, stream_id, s);
    if (st == GENP_OK && ce != cudaSuccess) {
        cudaGetLastError();
        st = GENP_ERR_CUDA;
    }
    if (st != GENP_OK) {
        free_multiplier(G);
        return st;
    }
    *out = G;
    return GENP_OK;
}

int genp_multiplier_side(genp_multiplier *G, int side) {
    if (!G || side < -1 || side > 1) return GENP_ERR_ARG;
    const int old = G->side;
    if (side >= 0) G->side = side;
    return old;
}

genp_status genp_redraw_multiplier(genp_multiplier *G, uint64_t seed, uint64_t stream_id, void *cuda_stream) {
    if (!G) return GENP_ERR_ARG;
    G->last_stream = S(cuda_stream);
    CU(draw_multiplier(G, seed, stream_id, S(cuda_stream)));
    return GENP_OK;
}

uint64_t genp_launch_count(void) {
    const volatile unsigned long long *b = g_body_launches;
    return g_launches.load(std::memory_order_relaxed) + (b ? *b : 0ull);
}

genp_status genp_gemm_bf16(int64_t m, int64_t n, int64_t K, float alpha, const void *A, int64_t lda, const void *Bt,
                           int64_t ldb, float beta, const float *Cin, int64_t ldci, float *D, int64_t ldd,
                           void *cuda_stream) {
    if (m < 0 || n < 0 || K < 1 || !A || !Bt || !D) return GENP_ERR_ARG;
    if (lda < K || ldb < K || ldd < n || (lda % 8) || (ldb % 8)) return GENP_ERR_ARG;
    if (((uintptr_t)A % 16) || ((uintptr_t)Bt % 16)) return GENP_ERR_ARG;
    if (beta != 0.0f && (!Cin || ldci < n)) return GENP_ERR_ARG;
    if (m > INT32_MAX || n > INT32_MAX || K > INT32_MAX || cdiv(m, 128) > 65535) return GENP_ERR_ARG;
    CU(tc_gemm_bf16(m, n, K, alpha, (const __nv_bfloat16 *)A, lda, (const __nv_bfloat16 *)Bt, ldb, beta, Cin, ldci, D,
                    ldd, nullptr, S(cuda_stream)));
    return GENP_OK;
}

genp_status genp_quantize_e4m3(const void *src, int64_t lds, genp_prec src_prec, int64_t m, int64_t K, int trans,
                               uint8_t *dst, int64_t ldq, float *scales, void *cuda_stream) {
    if (!src || !dst || !scales || m < 0 || K < 0) return GENP_ERR_ARG;
    if (src_prec != GENP_FP64 && src_prec != GENP_FP32) return GENP_ERR_ARG;
    if (m == 0 || K == 0) return GENP_OK;
    if (lds < (trans ? m : K) || ldq < K || (ldq % 16) || ((uintptr_t)dst % 16)) return GENP_ERR_ARG;
    if (m > INT32_MAX || K > INT32_MAX || cdiv(m, 128) > 65535) return GENP_ERR_ARG;
    cudaStream_t s = S(cuda_stream);
    if (src_prec == GENP_FP64)
        CU(quant_e4m3<double>(static_cast<const double *>(src), lds, m, K, trans != 0, dst, ldq, scales, s));
    else
        CU(quant_e4m3<float>(static_cast<const float *>(src), lds, m, K, trans != 0, dst, ldq, scales, s));
    return GENP_OK;
}

genp_status genp_gemm_e4m3(int64_t m, int64_t n, int64_t K, float alpha, const uint8_t *A, int64_t lda,
                           const float *scale_a, const uint8_t *Bt, int64_t ldb, const float *scale_b, float beta,
                           const float *Cin, int64_t ldci, float *D, int64_t ldd, void *cuda_stream) {
    if (m < 0 || n < 0 || K < 1 || !A || !Bt || !D || !scale_a || !scale_b) return GENP_ERR_ARG;
    if (lda < K || ldb < K || ldd < n || (lda % 16) || (ldb % 16)) return GENP_ERR_ARG;
    if (((uintptr_t)A % 16) || ((uintptr_t)Bt % 16)) return GENP_ERR_ARG;
    if (beta != 0.0f && (!Cin || ldci < n)) return GENP_ERR_ARG;
    if (m > INT32_MAX || n > INT32_MAX || K > 262144 || cdiv(m, 128) > 65535) return GENP_ERR_ARG;
    CU(tc_gemm_e4m3(m, n, K, alpha, A, lda, scale_a, Bt, ldb, scale_b, beta, Cin, ldci, D, ldd, S(cuda_stream)));
    return GENP_OK;
}

genp_status genp_profile_enable(int on) {
    tc_profile_enable(on != 0);
    return GENP_OK;
}

genp_status genp_profile_launches(double *ms, double *flops, int cap, int *launches) {
    if (!launches || cap < 0 || (cap > 0 && !ms && !flops)) return GENP_ERR_ARG;
    const int c = tc_profile_launches(ms, flops, cap);
    if (c < 0) return GENP_ERR_CUDA;
    *launches = c;
    return GENP_OK;
}

genp_status genp_profile_class(int cls, double *ms, double *work, int *launches) {
    if (!ms || !work || !launches || cls < kProfTensor || cls >= kProfClasses) return GENP_ERR_ARG;
    const int c = profile_class_read(cls, ms, work);
    if (c < 0) return GENP_ERR_CUDA;
    *launches = c;
    return GENP_OK;
}

genp_status genp_profile_read(double *ms, double *flops, int *launches) {
    if (!ms || !flops || !launches) return GENP_ERR_ARG;
    const int c = tc_profile_read(ms, flops);
    if (c < 0) return GENP_ERR_CUDA;
    *launches = c;
    return GENP_OK;
}

int genp_sliced_digits(int digits) {
    if (digits == 0) return sliced_digits();
    return set_sliced_digits(digits);
}

int genp_sliced_precondition_digits(int digits) {
    if (digits == 0) return sliced_precond_digits();
    return set_sliced_precond_digits(digits);
}

int genp_sliced_multiplier_digits(int digits) {
    if (digits == 0) return sliced_mult_digits();
    return set_sliced_mult_digits(digits);
}

genp_status genp_gemm_sliced(int64_t m, int64_t n, int64_t K, double alpha, const double *A, int64_t lda,
                             const double *B, int64_t ldb, double beta, double *D, int64_t ldd, int digits,
                             void *cuda_stream) {
    if (m < 0 || n < 0 || K < 1 || !A || !B || !D) return GENP_ERR_ARG;
    const int nd = digits == 0 ? sliced_digits() : digits;
    if (nd < 3 || nd > 7) return GENP_ERR_ARG;
    if (lda < K || ldb < n || ldd < n) return GENP_ERR_ARG;
    if (m > INT32_MAX || n > INT32_MAX || cdiv(m, 128) > 65535) return GENP_ERR_ARG;
    if (m == 0 || n == 0) return GENP_OK;
    cudaStream_t s = S(cuda_stream);
    keep_pool_cached();
    const int64_t ldq = kSlicedLdq, ldw = round8(n);
    const size_t wbytes = (size_t)m * ldw * 8, abytes = (size_t)m * ldq * 2, bbytes = (size_t)n * ldq * 2;
    char *buf = nullptr;
    if (cudaMallocAsync((void **)&buf, wbytes + abytes + bbytes + (size_t)(m + n) * sizeof(int) + 256, s) !=
        cudaSuccess) {
        cudaGetLastError();
        return GENP_ERR_NOMEM;
    }
    dfloat *W = reinterpret_cast<dfloat *>(buf);
    __nv_bfloat16 *Aq = reinterpret_cast<__nv_bfloat16 *>(buf + wbytes);
    __nv_bfloat16 *Bq = reinterpret_cast<__nv_bfloat16 *>(buf + wbytes + abytes);
    int *ex = reinterpret_cast<int *>(buf + wbytes + abytes + bbytes);
    cudaError_t e = sliced_matmul(nd, m, n, K, A, lda, B, ldb, W, ldw, Aq, Bq, ex, s);
    if (e == cudaSuccess) e = df_axpby(alpha, W, ldw, beta, D, ldd, m, n, s);
    cudaError_t f = cudaFreeAsync(buf, s);
    CU(e);
    CU(f);
    return GENP_OK;
}

genp_status genp_lowrank(int64_t m, int64_t n, const double *A, int64_t lda, int64_t r, genp_mult_kind kind,
                         uint64_t seed, uint64_t stream_id, double *G, int64_t ldg, double *Q, int64_t ldq, double *R,
                         int64_t ldr, double *AQ, int64_t ldaq, int *dev_status, void *cuda_stream) {
    if (m < 1 || n < 1 || !A || !Q || lda < n || r < 1 || r > n || r > 128) return GENP_ERR_ARG;
    if (kind != GENP_MULT_GAUSSIAN && kind != GENP_MULT_TOEPLITZ) return GENP_ERR_ARG;
    if (ldq < r || (G && ldg < r) || (R && ldr < r) || (AQ && ldaq < r)) return GENP_ERR_ARG;
    cudaStream_t s = S(cuda_stream);
    keep_pool_cached();
    void *work = nullptr;
    if (cudaMallocAsync(&work, lowrank_work_bytes(m, n, r), s) != cudaSuccess) {
        cudaGetLastError();
        return GENP_ERR_NOMEM;
    }
    if (dev_status) CU(cudaMemsetAsync(dev_status, 0, sizeof(int), s));
    cudaError_t e = lowrank_run(m, n, A, lda, r, kind == GENP_MULT_TOEPLITZ, seed, stream_id, G, ldg, Q, ldq, R, ldr,
                                AQ, ldaq, dev_status, work, s);
    cudaError_t f = cudaFreeAsync(work, s);
    CU(e);
    CU(f);
    return GENP_OK;
}

genp_status genp_numerical_rank(int64_t m, int64_t n, const double *A, int64_t lda, int64_t r_lo, int64_t r_hi,
                                double cond_max, uint64_t seed, uint64_t stream_id, int64_t *rank, double *B,
                                int64_t ldb, void *cuda_stream) {
    if (m < 1 || n < 1 || !A || !rank || lda < n) return GENP_ERR_ARG;
    if (r_lo < 0 || r_hi < r_lo || r_hi > n || r_hi > 128 || !(cond_max > 1.0)) return GENP_ERR_ARG;
    if (B && ldb < r_hi) return GENP_ERR_ARG;
    if (r_hi == 0) {
        *rank = 0;
        return GENP_OK;
    }
    cudaStream_t s = S(cuda_stream);
    keep_pool_cached();
    void *work = nullptr;
    if (cudaMallocAsync(&work, numerical_rank_work_bytes(m, n, r_hi), s) != cudaSuccess) {
        cudaGetLastError();
        return GENP_ERR_NOMEM;
    }
    double *hk = nullptr;
    if (cudaMallocHost((void **)&hk, sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeAsync(work, s);
        return GENP_ERR_NOMEM;
    }
    cudaError_t e = numerical_rank_run(m, n, A, lda, r_lo, r_hi, cond_max, seed, stream_id, rank, B, ldb, work, hk, s);
    cudaError_t f = cudaFreeAsync(work, s);
    if (f == cudaSuccess) f = cudaStreamSynchronize(s);
    cudaFreeHost(hk);
    CU(e);
    CU(f);
    return GENP_OK;
}

genp_status genp_device_check(int clear) {
    CU(cudaDeviceSynchronize());
    const int v = tc_timeout_flag(clear != 0), w = solve_timeout_flag(clear != 0);
    if (v < 0 || w < 0) return GENP_ERR_CUDA;
    return (v || w) ? GENP_ERR_TIMEOUT : GENP_OK;
}

genp_status genp_multiplier_export(const genp_multiplier *G, double *dense, int64_t ldd, double *first_col,
                                   int32_t *rows, int8_t *signs, void *cuda_stream) {
    if (!G) return GENP_ERR_ARG;
    if (dense && ldd < G->n) return GENP_ERR_ARG;
    if (first_col && G->kind != GENP_MULT_CIRCULANT && G->kind != GENP_MULT_HOUSEHOLDER_PM1) return GENP_ERR_ARG;
    if ((rows || signs) && G->kind != GENP_MULT_SPARSE_PM1) return GENP_ERR_ARG;
    cudaStream_t s = S(cuda_stream);
    const int64_t n = G->n;
    if (dense) {
        if (G->kind == GENP_MULT_GAUSSIAN)
            CU(cudaMemcpy2DAsync(dense, ldd * sizeof(double), G->dense, n * sizeof(double), n * sizeof(double), n,
                                 cudaMemcpyDeviceToDevice, s));
        else if (G->kind == GENP_MULT_CIRCULANT)
            CU(launch_circulant_to_dense(G->g, G->cn, n, dense, ldd, s));
        else if (G->kind == GENP_MULT_HOUSEHOLDER_PM1)
            CU(house_to_dense(G, dense, ldd, s));
        else if (G->kind == GENP_MULT_IDENTITY) {
            note_launch();
            k_eye<<<dim3((unsigned)cdiv(n < 2048 ? n : 2048, 256), (unsigned)(n < 65535 ? n : 65535)), 256, 0, s>>>(
                dense, n, ldd);
            CU(cudaGetLastError());
        } else
            CU(launch_sparse_to_dense(G->rows, G->signs, n, G->nnz, dense, ldd, s));
    }
    if (first_col)
        CU(cudaMemcpyAsync(first_col, G->g, (G->kind == GENP_MULT_CIRCULANT ? G->cn : n) * sizeof(double),
                           cudaMemcpyDeviceToDevice, s));
    if (rows) CU(cudaMemcpyAsync(rows, G->rows, (size_t)n * G->nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    if (signs) CU(cudaMemcpyAsync(signs, G->signs, (size_t)n * G->nnz, cudaMemcpyDeviceToDevice, s));
    return GENP_OK;
}

genp_status genp_multiplier_query(const genp_multiplier *G, int64_t *n, int *kind, int *nnz_per_col) {
    if (!G) return GENP_ERR_ARG;
    if (n) *n = G->n;
    if (kind)
        *kind = G->pm1 ? (int)GENP_MULT_CIRCULANT_PM1 : G->toeplitz ? (int)GENP_MULT_TOEPLITZ : (int)G->kind;
    if (nnz_per_col) *nnz_per_col = G->nnz;
    return GENP_OK;
}

void genp_multiplier_destroy(genp_multiplier *G) {
    if (G) free_multiplier(G);
}

genp_status genp_precondition(const genp_multiplier *G, const void *A, int64_t lda, genp_prec a_prec, void *C,
                              int64_t ldc, genp_prec c_prec, void *cuda_stream) {
    keep_pool_cached();
    if (!G || !A || !C) return GENP_ERR_ARG;
    const int64_t n = G->n;
    if (lda < n || ldc < n) return GENP_ERR_ARG;
    if (a_prec != GENP_FP64 && a_prec != GENP_FP32) return GENP_ERR_ARG;
    if (!factor_prec_ok(c_prec)) return GENP_ERR_ARG;
    if (f64_factors(c_prec) && a_prec != GENP_FP64) return GENP_ERR_ARG;
    cudaStream_t s = S(cuda_stream);
    if (G->kind == GENP_MULT_IDENTITY) {   // plain GENP: C = A in the factor's storage type
        if (f64_factors(c_prec))
            CU((convert_matrix<double, double>(static_cast<const double *>(A), lda, static_cast<double *>(C), ldc, n, n,
                                               nullptr, s)));
        else if (a_prec == GENP_FP64)
            CU((convert_matrix<double, float>(static_cast<const double *>(A), lda, static_cast<float *>(C), ldc, n, n,
                                              nullptr, s)));
        else
            CU((convert_matrix<float, float>(static_cast<const float *>(A), lda, static_cast<float *>(C), ldc, n, n,
                                             nullptr, s)));
        return GENP_OK;
    }
    if (G->side == GENP_SIDE_LEFT) {
        // C = G A (Cor. 4.1's GM half): the multiplier's product with the
        // columns of A, as for X = G Y with n right-hand sides
        if (a_prec != GENP_FP64 || tc_prec(c_prec)) return GENP_ERR_UNSUPPORTED;
        const double *a = static_cast<const double *>(A);
        if (c_prec == GENP_BF16_SLICED && G->kind == GENP_MULT_GAUSSIAN) {
            const int nd = sliced_precond_digits();
            // G on the sliced grid is exact in its one or two digits: nd or 2 nd - 1
            // digit products instead of nd (nd + 1) / 2
            const int ndg = (G->grid == GENP_BF16_SLICED && nd >= 5) ? G->grid_digits : nd;
            const int64_t ldq = (int64_t)nd * (ndg <= 2 ? kSlicedChunk2 : kSlicedChunk), ldd = round8(n);
            char *buf = nullptr;
            const size_t dbytes = (size_t)n * ldd * 8, qbytes = (size_t)n * ldq * sizeof(__nv_bfloat16);
            CU(cudaMallocAsync((void **)&buf, dbytes + 2 * qbytes + (size_t)2 * n * sizeof(int) + 256, s));
            dfloat *D = reinterpret_cast<dfloat *>(buf);
            __nv_bfloat16 *Aq = reinterpret_cast<__nv_bfloat16 *>(buf + dbytes);
            __nv_bfloat16 *Bq = Aq + (size_t)n * ldq;
            int *ex = reinterpret_cast<int *>(Bq + (size_t)n * ldq);
            CU(sliced_matmul(ndg, n, n, n, G->dense, n, a, lda, D, ldd, Aq, Bq, ex, s, nd));
            CU(df_to_f64(D, ldd, static_cast<double *>(C), ldc, n, n, s));
            CU(cudaFreeAsync(buf, s));
            return GENP_OK;
        }
        if (f64_factors(c_prec)) {
            CU(apply_multiplier(G, false, a, lda, static_cast<double *>(C), ldc, n, false, nullptr, s));
            return GENP_OK;
        }
        double *tmp = nullptr;   // FP32 factors: the FP64 product, rounded once
        CU(cudaMallocAsync((void **)&tmp, (size_t)n * n * sizeof(double), s));
        CU(apply_multiplier(G, false, a, lda, tmp, n, n, false, nullptr, s));
        CU((convert_matrix<double, float>(tmp, n, static_cast<float *>(C), ldc, n, n, nullptr, s)));
        CU(cudaFreeAsync(tmp, s));
        return GENP_OK;
    }
    if (c_prec == GENP_BF16_SLICED && G->kind == GENP_MULT_GAUSSIAN) {
        // C = A G on the BF16 tensor cores from exact digit slices (as many
        // digits as genp_sliced_precondition_digits asks), summed in
        // double-float and rounded to FP64 once.
        const int nd = sliced_precond_digits();
        // G on the sliced grid is exact in its one or two digits: nd or 2 nd - 1
        // digit products instead of nd (nd + 1) / 2
        const int ndg = (G->grid == GENP_BF16_SLICED && nd >= 5) ? G->grid_digits : nd;
        const int64_t ldq = (int64_t)nd * (ndg <= 2 ? kSlicedChunk2 : kSlicedChunk), ldd = round8(n);
        char *buf = nullptr;
        const size_t dbytes = (size_t)n * ldd * 8, qbytes = (size_t)n * ldq * sizeof(__nv_bfloat16);
        CU(cudaMallocAsync((void **)&buf, dbytes + 2 * qbytes + (size_t)2 * n * sizeof(int) + 256, s));
        dfloat *D = reinterpret_cast<dfloat *>(buf);
        __nv_bfloat16 *Aq = reinterpret_cast<__nv_bfloat16 *>(buf + dbytes);
        __nv_bfloat16 *Bq = Aq + (size_t)n * ldq;
        int *ex = reinterpret_cast<int *>(Bq + (size_t)n * ldq);
        if (ndg <= 2) {
            // G (one or two digits) on the M side, A's rows (nd digits) along N:
            // the product comes out transposed and is turned around on the way to FP64
            CU(sliced_matmul_t(nd, ndg, n, n, n, static_cast<const double *>(A), lda, G->dense, n, D, ldd, Bq, Aq,
                               ex, s));
            CU(df_to_f64_T(D, ldd, static_cast<double *>(C), ldc, n, n, s));
        } else {
            CU(sliced_matmul(nd, n, n, n, static_cast<const double *>(A), lda, G->dense, n, D, ldd, Aq, Bq, ex, s));
            CU(df_to_f64(D, ldd, static_cast<double *>(C), ldc, n, n, s));
        }
        CU(cudaFreeAsync(buf, s));
        return GENP_OK;
    }
    if (c_prec == GENP_BF16_SLICED) c_prec = GENP_FP64;   // circulant / sparse products: FP64 FFT / gather
    if (c_prec == GENP_FP8_E4M3 && G->kind == GENP_MULT_GAUSSIAN) {
        // Tensor cores, e4m3: C = A_q G with A_q the tile-scaled e4m3 codes of
        // A; G is on the FP8 grid, so its tile-scaled codes are exact.
        if (G->grid != GENP_FP8_E4M3) return GENP_ERR_ARG;
        const int64_t ldq = (n + 15) / 16 * 16, tiles = e4m3_tiles(n, n);
        char *buf = nullptr;
        const size_t qbytes = align256((size_t)n * ldq);
        CU(cudaMallocAsync((void **)&buf, 2 * qbytes + 2 * (size_t)tiles * sizeof(float), s));
        uint8_t *Aq = reinterpret_cast<uint8_t *>(buf), *Gq = Aq + qbytes;
        float *sA = reinterpret_cast<float *>(Gq + qbytes), *sG = sA + tiles;
        if (a_prec == GENP_FP64)
            CU(quant_e4m3<double>(static_cast<const double *>(A), lda, n, n, false, Aq, ldq, sA, s));
        else
            CU(quant_e4m3<float>(static_cast<const float *>(A), lda, n, n, false, Aq, ldq, sA, s));
        CU(quant_e4m3<double>(G->dense, n, n, n, true, Gq, ldq, sG, s));   // rows of G^T
        CU(tc_gemm_e4m3(n, n, n, 1.0f, Aq, ldq, sA, Gq, ldq, sG, 0.0f, nullptr, 0, static_cast<float *>(C), ldc, s));
        CU(cudaFreeAsync(buf, s));
        return GENP_OK;
    }
    if (tc_prec(c_prec) && c_prec != GENP_FP8_E4M3 && G->kind == GENP_MULT_GAUSSIAN) {
        // Tensor cores: C = sum_t a_t G over the BF16 terms a_t of A (one term
        // for BF16, three for BF16X3); G is exact on the BF16 grid.
        if (!G->dense_bf16) return GENP_ERR_ARG;
        const int terms = c_prec == GENP_BF16X3 ? 3 : 1;
        const int64_t ldq = round8(n);
        __nv_bfloat16 *buf = nullptr;
        CU(cudaMallocAsync((void **)&buf, (size_t)n * ldq * sizeof(__nv_bfloat16), s));
        float *c = static_cast<float *>(C);
        for (int t = 0; t < terms; ++t) {
            if (a_prec == GENP_FP64)
                CU(split_rows<double>((const double *)A, lda, n, n, buf, ldq, 1, true, t, s));
            else
                CU(split_rows<float>((const float *)A, lda, n, n, buf, ldq, 1, true, t, s));
            CU(tc_gemm_bf16(n, n, n, 1.0f, buf, ldq, G->dense_bf16, round8(n), t > 0 ? 1.0f : 0.0f, c, ldc, c, ldc,
                            nullptr, s));
        }
        CU(cudaFreeAsync(buf, s));
        return GENP_OK;
    }
    if (tc_prec(c_prec)) c_prec = GENP_FP32;  // circulant and sparse products run in FP32 (FFT / exact gather)
    if (c_prec == GENP_FP64) {
        const double *a = static_cast<const double *>(A);
        double *c = static_cast<double *>(C);
        switch (G->kind) {
            case GENP_MULT_GAUSSIAN:
                CU(gemm<double>(n, n, n, 1.0, a, lda, false, G->dense, n, 0.0, nullptr, 0, c, ldc, nullptr, s));
                break;
            case GENP_MULT_CIRCULANT:
                if (circ_fft_supported(G->cn)) {
                    // algorithmic bytes: A read and C written once (16 n^2)
                    auto *ev = profile_class_slot(kProfPrecond, 16.0 * (double)n * (double)n);
                    prof_begin(ev, s);
                    CU((circ_apply<double, double>(G, 0, a, lda, 1, c, ldc, 1, n, nullptr, s)));
                    prof_end(ev, s);
                } else {
                    CU((circ_matmul_direct<double, double>(G->g, G->cn, n, a, lda, c, ldc, s)));
                }
                break;
            case GENP_MULT_SPARSE_PM1: {
                // algorithmic bytes: A read and C written once (16 n^2; the indices are 5 nnz n)
                auto *ev = profile_class_slot(kProfPrecond, 16.0 * (double)n * (double)n);
                prof_begin(ev, s);
                CU((sparse_precondition<double, double>(G, a, lda, c, ldc, s)));
                prof_end(ev, s);
                break;
            }
            case GENP_MULT_HOUSEHOLDER_PM1: CU((house_precondition<double, double>(G, a, lda, c, ldc, s))); break;
            default: return GENP_ERR_ARG;
        }
        return GENP_OK;
    }
    // FP32 factorization: C (float) = A G in FP32 arithmetic.
    float *c = static_cast<float *>(C);
    if (G->kind == GENP_MULT_SPARSE_PM1) {
        if (a_prec == GENP_FP64) CU((sparse_precondition<double, float>(G, (const double *)A, lda, c, ldc, s)));
        else CU((sparse_precondition<float, float>(G, (const float *)A, lda, c, ldc, s)));
        return GENP_OK;
    }
    if (G->kind == GENP_MULT_HOUSEHOLDER_PM1) {
        if (a_prec == GENP_FP64) CU((house_precondition<double, float>(G, (const double *)A, lda, c, ldc, s)));
        else CU((house_precondition<float, float>(G, (const float *)A, lda, c, ldc, s)));
        return GENP_OK;
    }
    if (G->kind == GENP_MULT_CIRCULANT && circ_fft_supported(G->cn)) {
        if (a_prec == GENP_FP64) CU((circ_apply<double, float>(G, 0, (const double *)A, lda, 1, c, ldc, 1, n, nullptr, s)));
        else CU((circ_apply<float, float>(G, 0, (const float *)A, lda, 1, c, ldc, 1, n, nullptr, s)));
        return GENP_OK;
    }
    if (G->kind == GENP_MULT_GAUSSIAN && !G->dense_f32) return GENP_ERR_ARG;  // needs an FP32-exact G
    const float *a32 = static_cast<const float *>(A);
    int64_t lda32 = lda;
    float *tmp = nullptr;
    if (a_prec == GENP_FP64) {
        CU(cudaMallocAsync((void **)&tmp, (size_t)n * n * sizeof(float), s));
        CU((convert_matrix<double, float>((const double *)A, lda, tmp, n, n, n, nullptr, s)));
        a32 = tmp;
        lda32 = n;
    }
    if (G->kind == GENP_MULT_GAUSSIAN)
        CU(gemm<float>(n, n, n, 1.0f, a32, lda32, false, G->dense_f32, n, 0.0f, nullptr, 0, c, ldc, nullptr, s));
    else
        CU((circ_matmul_direct<float, float>(G->g, G->cn, n, a32, lda32, c, ldc, s)));
    if (tmp) CU(cudaFreeAsync(tmp, s));
    return GENP_OK;
}

namespace {
genp_status new_factors(void *C, int64_t n, int64_t ldc, genp_prec prec, int64_t nb, bool block, cudaStream_t s,
                        genp_factors **out);
}

genp_status genp_factor(void *C, int64_t n, int64_t ldc, genp_prec prec, int64_t nb, void *cuda_stream,
                        genp_factors **out) {
    if (!out) return GENP_ERR_ARG;
    *out = nullptr;
    if (!C || n < 1 || n > 2147483647LL || ldc < n) return GENP_ERR_ARG;
    if (!factor_prec_ok(prec)) return GENP_ERR_ARG;
    if (nb == 0) nb = (tc_prec(prec) || prec == GENP_BF16_SLICED) ? 128 : 64;
    if (nb < 1 || nb > 128) return GENP_ERR_ARG;
    return new_factors(C, n, ldc, prec, nb, false, S(cuda_stream), out);
}

genp_status genp_block_factor(double *C, int64_t n, int64_t ldc, int64_t nb, void *cuda_stream,
                              genp_factors **out) {
    if (!out) return GENP_ERR_ARG;
    *out = nullptr;
    if (!C || n < 1 || n > 2147483647LL || ldc < n) return GENP_ERR_ARG;
    if (nb == 0) nb = 64;
    if (nb != 64) return GENP_ERR_UNSUPPORTED;
    return new_factors(C, n, ldc, GENP_FP64, nb, true, S(cuda_stream), out);
}

namespace {
genp_status new_factors(void *C, int64_t n, int64_t ldc, genp_prec prec, int64_t nb, bool block, cudaStream_t s,
                        genp_factors **out) {
    genp_factors *F = new (std::nothrow) genp_factors();
    if (!F) return GENP_ERR_NOMEM;
    F->block = block;
    F->C = C;
    F->n = n;
    F->ldc = ldc;
    F->nb = nb;
    F->prec = prec;
    F->last_stream = s;
    genp_status st = dalloc(&F->st, 1);
    if (st == GENP_OK) st = dalloc(&F->norms, 2);
    if (st == GENP_OK) st = dalloc(&F->trsv_sync, (size_t)trsv_sync_ints(n));
    if (st == GENP_OK) {
        if (f64_factors(prec)) st = dalloc(reinterpret_cast<double **>(&F->trsv_y), (size_t)trsv_y_elems(n));
        else st = dalloc(reinterpret_cast<float **>(&F->trsv_y), (size_t)trsv_y_elems(n));
    }
    if (st == GENP_OK) {
        if (f64_factors(prec)) st = dalloc(reinterpret_cast<double **>(&F->dinv), (size_t)diag_inverse_elems(n));
        else st = dalloc(reinterpret_cast<float **>(&F->dinv), (size_t)diag_inverse_elems(n));
    }
    if (st == GENP_OK && tc_prec(prec)) {
        F->tc_ldq = round8(nb * split_terms(prec));
        st = dalloc(&F->tcA, (size_t)n * F->tc_ldq);
        if (st == GENP_OK) st = dalloc(&F->tcB, (size_t)n * F->tc_ldq);
        if (st == GENP_OK && prec == GENP_FP8_E4M3) st = dalloc(&F->qscale, (size_t)2 * cdiv(n, 128));
    }
    if (st == GENP_OK && prec == GENP_BF16_SLICED) {
        F->nd = sliced_digits();
        F->tc_ldq = (int64_t)F->nd * sliced_kpad(2 * nb > kSlicedOuter ? 2 * nb : kSlicedOuter);   // outer steps
        F->ldw = round8(n);   // 16-byte aligned rows for the vectorized epilogue
        st = dalloc(&F->tcA, (size_t)n * F->tc_ldq);
        if (st == GENP_OK) st = dalloc(&F->tcB, (size_t)n * F->tc_ldq);
        if (st == GENP_OK) st = dalloc(reinterpret_cast<double **>(&F->W), (size_t)n * F->ldw);
        // + the inner-dimension keys (8 B each) of an outer step
        if (st == GENP_OK) st = dalloc(&F->exps, (size_t)(2 * n + 2 * (2 * nb > kSlicedOuter ? 2 * nb : kSlicedOuter)));
        // the inverses, then the masked diagonal blocks, as double-float pairs
        if (st == GENP_OK) st = dalloc(reinterpret_cast<double **>(&F->dinv_df), (size_t)(2 * diag_inverse_elems(n)));
    }
    if (st == GENP_OK && cudaMallocHost(&F->host_info, sizeof(DevStatus)) != cudaSuccess) {
        cudaGetLastError();
        F->host_info = nullptr;
        st = GENP_ERR_NOMEM;
    }
    if (st == GENP_OK && cudaMemsetAsync(F->st, 0, sizeof(DevStatus), s) != cudaSuccess) st = GENP_ERR_CUDA;
    if (st == GENP_OK && cudaMemsetAsync(F->norms, 0, 2 * sizeof(DevNorms), s) != cudaSuccess) st = GENP_ERR_CUDA;
    if (st == GENP_OK && factor_run(F, s) != cudaSuccess) st = GENP_ERR_CUDA;
    if (st != GENP_OK) {
        cudaGetLastError();
        genp_factors_destroy(F);
        return st;
    }
    *out = F;
    return GENP_OK;
}
}  // namespace

genp_status genp_refactor(genp_factors *F, void *C, int64_t ldc, void *cuda_stream) {
    if (!F || !C || ldc < F->n) return GENP_ERR_ARG;
    F->C = C;
    F->ldc = ldc;
    F->last_stream = S(cuda_stream);
    CU(factor_run(F, S(cuda_stream)));
    return GENP_OK;
}

void genp_factors_destroy(genp_factors *F) {
    if (!F) return;
    bool any = F->rg_stream != nullptr || F->la_stream != nullptr;
    for (auto &g : F->rgraph) any = any || g.exec;
    if (any) cudaDeviceSynchronize();   // graphs and their streams may still be in use
    for (auto &g : F->rgraph) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        cudaFree(g.body_counts);
    }
    if (F->rg_stream) cudaStreamDestroy(F->rg_stream);
    for (auto &b : F->rg_body)
        if (b) cudaStreamDestroy(b);
    if (F->la_stream) cudaStreamDestroy(F->la_stream);
    for (auto &ev : F->la_ev)
        if (ev) cudaEventDestroy(ev);
    cudaFree(F->st);
    cudaFree(F->norms);
    cudaFree(F->work);
    cudaFree(F->tcA);
    cudaFree(F->tcB);
    cudaFree(F->qscale);
    cudaFree(F->W);
    cudaFree(F->exps);
    cudaFree(F->trsv_sync);
    cudaFree(F->trsv_y);
    cudaFree(F->dinv);
    cudaFree(F->dinv_df);
    if (F->host_info) cudaFreeHost(F->host_info);
    delete F;
}

genp_status genp_solve(const genp_factors *F, const genp_multiplier *G, const double *B, int64_t ldb, int64_t nrhs,
                       double *X, int64_t ldx, void *cuda_stream) {
    if (!F || !G || !B || !X) return GENP_ERR_ARG;
    if (G->n != F->n || nrhs < 1 || ldb < nrhs || ldx < nrhs) return GENP_ERR_ARG;
    if (X == B && ldx != ldb) return GENP_ERR_ARG;
    cudaStream_t s = S(cuda_stream);
    genp_factors *Fm = const_cast<genp_factors *>(F);
    const int64_t n = F->n;
    const size_t yd = align256((size_t)n * nrhs * sizeof(double)), yf = align256((size_t)n * nrhs * sizeof(float));
    TRY(ensure_work(Fm, yd + yf, s));
    double *Y = static_cast<double *>(F->work);
    float *Yf = reinterpret_cast<float *>(static_cast<char *>(F->work) + yd);
    const bool left = G->side == GENP_SIDE_LEFT;
    if (left) CU(apply_multiplier(G, false, B, ldb, Y, nrhs, nrhs, false, nullptr, s));   // G B
    else CU((convert_matrix<double, double>(B, ldb, Y, nrhs, n, nrhs, nullptr, s)));
    if (f64_factors(F->prec)) {
        CU(lu_solve_inplace<double>(F, Y, nrhs, nrhs, false, nullptr, s));
    } else {
        CU((convert_matrix<double, float>(Y, nrhs, Yf, nrhs, n, nrhs, nullptr, s)));
        CU(lu_solve_inplace<float>(F, Yf, nrhs, nrhs, false, nullptr, s));
        CU((convert_matrix<float, double>(Yf, nrhs, Y, nrhs, n, nrhs, nullptr, s)));
    }
    if (left) CU((convert_matrix<double, double>(Y, nrhs, X, ldx, n, nrhs, nullptr, s)));
    else CU(apply_multiplier(G, false, Y, nrhs, X, ldx, nrhs, false, nullptr, s));
    Fm->last_stream = s;
    return GENP_OK;
}

namespace {

bool g_refine_graphs = true;

// The launch sequence of genp_refine (workspace already in place).
genp_status refine_enqueue(const double *A, int64_t lda, genp_factors *Fm, const genp_multiplier *G,
                           const double *B, int64_t ldb, int64_t nrhs, double *X, int64_t ldx, double tol,
                           int max_iter, int method, cudaStream_t s, CondRec *cr = nullptr) {
    const genp_factors *F = Fm;
    const int64_t n = F->n;
    if (method == 1) {
        CU(refine_gmres(Fm, G, A, lda, B, ldb, nrhs, X, ldx, tol, max_iter, F->work, s, cr));
        return GENP_OK;
    }
    const size_t rd = align256((size_t)n * nrhs * sizeof(double));
    double *R = static_cast<double *>(F->work);
    double *T = reinterpret_cast<double *>(static_cast<char *>(F->work) + rd);
    float *Rf = reinterpret_cast<float *>(static_cast<char *>(F->work) + 2 * rd);
    const int *done = &F->st->refine_done;
    const bool left = G->side == GENP_SIDE_LEFT;
    CU(refine_init(Fm, A, lda, n, s));
    for (int it = 0; it <= max_iter; ++it) {
        // the residual and its check, then the correction: each skipped once
        // the refinement has converged
        if (it > 0) CU(cond_begin(cr, s, done));
        CU(gemm<double>(n, nrhs, n, -1.0, A, lda, false, X, ldx, 1.0, B, ldb, R, nrhs, done, s));
        CU(refine_check(Fm, R, nrhs, X, ldx, B, ldb, n, nrhs, it, tol, max_iter, 1, s));
        if (it > 0) CU(cond_end(cr, s));
        if (it == max_iter) break;
        CU(cond_begin(cr, s, done));
        double *D = R;
        if (left) {   // d = U^-1 L^-1 (G r)
            CU(apply_multiplier(G, false, R, nrhs, T, nrhs, nrhs, false, done, s));
            D = T;
        }
        if (f64_factors(F->prec)) {
            CU(lu_solve_inplace<double>(F, D, nrhs, nrhs, false, done, s));
        } else {
            CU((convert_matrix<double, float>(D, nrhs, Rf, nrhs, n, nrhs, done, s)));
            CU(lu_solve_inplace<float>(F, Rf, nrhs, nrhs, false, done, s));
            CU((convert_matrix<float, double>(Rf, nrhs, D, nrhs, n, nrhs, done, s)));
        }
        if (left) CU(add_into(D, nrhs, X, ldx, n, nrhs, done, s));
        else CU(apply_multiplier(G, false, R, nrhs, X, ldx, nrhs, true, done, s));
        CU(cond_end(cr, s));
    }
    return GENP_OK;
}

// Records the refinement's launches on the factors' private stream into a
// CUDA graph; returns the instantiated graph in *exec and the kernels it
// holds in *launches.
genp_status refine_record(const double *A, int64_t lda, genp_factors *F, const genp_multiplier *G, const double *B,
                          int64_t ldb, int64_t nrhs, double *X, int64_t ldx, double tol, int max_iter, int method,
                          cudaGraphExec_t *exec, uint64_t *launches, int **body_counts) {
    if (!F->rg_stream && cudaStreamCreateWithFlags(&F->rg_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        F->rg_stream = nullptr;
        return GENP_ERR_CUDA;
    }
    for (auto &b : F->rg_body)
        if (!b && cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            b = nullptr;
            return GENP_ERR_CUDA;
        }
    {
        std::lock_guard<std::mutex> lk(g_body_launches_mu);
        if (!g_body_launches) {
            void *h = nullptr, *d = nullptr;
            if (cudaHostAlloc(&h, sizeof(unsigned long long), cudaHostAllocMapped) != cudaSuccess ||
                cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
                if (h) cudaFreeHost(h);
                cudaGetLastError();
                return GENP_ERR_CUDA;
            }
            *static_cast<unsigned long long *>(h) = 0;
            g_body_launches_dev = static_cast<unsigned long long *>(d);
            g_body_launches = static_cast<unsigned long long *>(h);
        }
    }
    if (!*body_counts) TRY(dalloc(body_counts, CondRec::kMaxBodies));
    CondRec cr;
    cr.chain[0] = F->rg_stream;
    cr.chain[1] = F->rg_body[0];
    cr.chain[2] = F->rg_body[1];
    cr.dev_counts = *body_counts;
    cudaStream_t rs = F->rg_stream;
    if (cudaStreamBeginCapture(rs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return GENP_ERR_CUDA;
    }
    const uint64_t l0 = g_launches.load(std::memory_order_relaxed);
    profile_suspend(true);
    genp_status st = refine_enqueue(A, lda, F, G, B, ldb, nrhs, X, ldx, tol, max_iter, method, rs, &cr);
    profile_suspend(false);
    while (cr.depth > 0) {   // a body left open by an error
        cudaGraph_t body = nullptr;
        cudaStreamEndCapture(cr.chain[cr.depth--], &body);
        if (st == GENP_OK) st = GENP_ERR_CUDA;
    }
    const uint64_t total = g_launches.load(std::memory_order_relaxed) - l0;
    *launches = total - cr.nested[0];
    g_launches.fetch_sub(total, std::memory_order_relaxed);   // counted when the graph runs
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(rs, &graph);
    if (st != GENP_OK || ec != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return st != GENP_OK ? st : GENP_ERR_CUDA;
    }
    if (!cr.counts.empty() && cudaMemcpy(*body_counts, cr.counts.data(), cr.counts.size() * sizeof(int),
                                         cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGraphDestroy(graph);
        cudaGetLastError();
        return GENP_ERR_CUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        *exec = nullptr;
        return GENP_ERR_CUDA;
    }
    return GENP_OK;
}

}  // namespace

int genp_refine_graphs(int enable) {
    const int old = g_refine_graphs ? 1 : 0;
    if (enable >= 0) g_refine_graphs = enable != 0;
    return old;
}

genp_status genp_refine(const double *A, int64_t lda, const genp_factors *F, const genp_multiplier *G, const double *B,
                        int64_t ldb, int64_t nrhs, double *X, int64_t ldx, double tol, int max_iter, int method,
                        void *cuda_stream) {
    if (!A || !F || !G || !B || !X) return GENP_ERR_ARG;
    const int64_t n = F->n;
    if (G->n != n || lda < n || nrhs < 1 || ldb < nrhs || ldx < nrhs) return GENP_ERR_ARG;
    if (max_iter < 0 || max_iter > GENP_MAX_REFINE || !(tol >= 0.0)) return GENP_ERR_ARG;
    if (method != 0 && method != 1) return GENP_ERR_ARG;
    if (nrhs > kMaxRhsChunk) return GENP_ERR_UNSUPPORTED;
    cudaStream_t s = S(cuda_stream);
    genp_factors *Fm = const_cast<genp_factors *>(F);
    if (method == 1) {
        TRY(ensure_work(Fm, gmres_work_bytes(n, nrhs), s));
    } else {
        const size_t rd = align256((size_t)n * nrhs * sizeof(double)),
                     yf = align256((size_t)n * nrhs * sizeof(float));
        TRY(ensure_work(Fm, 2 * rd + yf, s));
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        cap = cudaStreamCaptureStatusActive;   // unknown: take the plain path
    }
    if (!g_refine_graphs || cap != cudaStreamCaptureStatusNone) {
        // enqueued launch by launch (a caller capturing its own graph gets them in it)
        const genp_status st = refine_enqueue(A, lda, Fm, G, B, ldb, nrhs, X, ldx, tol, max_iter, method, s);
        if (st == GENP_OK) Fm->last_stream = s;
        return st;
    }
    double tolv = tol;
    uint64_t tolbits = 0;
    memcpy(&tolbits, &tolv, sizeof(tolbits));
    const uint64_t key[16] = {(uint64_t)(uintptr_t)A, (uint64_t)lda, (uint64_t)(uintptr_t)G, (uint64_t)(uintptr_t)B,
                              (uint64_t)ldb, (uint64_t)nrhs, (uint64_t)(uintptr_t)X, (uint64_t)ldx, tolbits,
                              (uint64_t)max_iter, (uint64_t)method, (uint64_t)G->side, (uint64_t)(uintptr_t)F->C,
                              (uint64_t)F->ldc, (uint64_t)(uintptr_t)F->work, 1};
    GenpRefineGraph *hit = nullptr;
    for (auto &g : Fm->rgraph)
        if (g.exec && memcmp(g.key, key, sizeof(key)) == 0) hit = &g;
    if (!hit) {
        GenpRefineGraph &slot = Fm->rgraph[Fm->rg_next];
        Fm->rg_next = (Fm->rg_next + 1) % 4;
        if (slot.exec) {
            // the slot's graph may still be queued on some stream: free it only
            // once everything enqueued so far has finished
            cudaDeviceSynchronize();
            cudaGraphExecDestroy(slot.exec);
            slot.exec = nullptr;
        }
        // the recording stream must see the caller's stream state (buffers
        // written by earlier calls): recording enqueues nothing, so no wait
        TRY(refine_record(A, lda, Fm, G, B, ldb, nrhs, X, ldx, tol, max_iter, method, &slot.exec, &slot.launches,
                          &slot.body_counts));
        memcpy(slot.key, key, sizeof(key));
        hit = &slot;
    }
    CU(cudaGraphLaunch(hit->exec, s));
    note_launches(hit->launches);
    Fm->last_stream = s;
    return GENP_OK;
}

genp_status genp_adjoint(const genp_factors *F, const genp_multiplier *G, const double *gX, int64_t ldg,
                         const double *X, int64_t ldx, int64_t nrhs, void *dA, int64_t ldda, double *dB, int64_t lddb,
                         void *cuda_stream) {
    if (!F || !G || !gX) return GENP_ERR_ARG;
    const int64_t n = F->n;
    if (G->n != n || nrhs < 1 || ldg < nrhs) return GENP_ERR_ARG;
    if (dA && (!X || ldx < nrhs || ldda < n)) return GENP_ERR_ARG;
    if (dB && lddb < nrhs) return GENP_ERR_ARG;
    cudaStream_t s = S(cuda_stream);
    genp_factors *Fm = const_cast<genp_factors *>(F);
    const size_t ld = align256((size_t)n * nrhs * sizeof(double)), yf = align256((size_t)n * nrhs * sizeof(float));
    TRY(ensure_work(Fm, 2 * ld + yf, s));
    double *Lam = static_cast<double *>(F->work);
    double *T = reinterpret_cast<double *>(static_cast<char *>(F->work) + ld);
    float *Lf = reinterpret_cast<float *>(static_cast<char *>(F->work) + 2 * ld);
    const bool left = G->side == GENP_SIDE_LEFT;
    // right: Lambda = L^-T U^-T (G^T gX);  left: Lambda = G^T (L^-T U^-T gX)
    double *Z = left ? T : Lam;
    if (left) CU((convert_matrix<double, double>(gX, ldg, Z, nrhs, n, nrhs, nullptr, s)));
    else CU(apply_multiplier(G, true, gX, ldg, Z, nrhs, nrhs, false, nullptr, s));
    if (f64_factors(F->prec)) {
        CU(lu_solve_inplace<double>(F, Z, nrhs, nrhs, true, nullptr, s));
    } else {
        CU((convert_matrix<double, float>(Z, nrhs, Lf, nrhs, n, nrhs, nullptr, s)));
        CU(lu_solve_inplace<float>(F, Lf, nrhs, nrhs, true, nullptr, s));
        CU((convert_matrix<float, double>(Lf, nrhs, Z, nrhs, n, nrhs, nullptr, s)));
    }
    if (left) CU(apply_multiplier(G, true, T, nrhs, Lam, nrhs, nrhs, false, nullptr, s));
    if (dB) CU((convert_matrix<double, double>(Lam, nrhs, dB, lddb, n, nrhs, nullptr, s)));
    if (dA) CU(outer_update(Lam, nrhs, X, ldx, n, nrhs, dA, ldda, !f64_factors(F->prec), s));
    Fm->last_stream = s;
    return GENP_OK;
}

genp_status genp_info_fetch(const genp_factors *F, genp_info *out, void *cuda_stream) {
    if (!F || !out) return GENP_ERR_ARG;
    cudaStream_t s = S(cuda_stream);
    CU(cudaMemcpyAsync(F->host_info, F->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    DevStatus h;
    memcpy(&h, F->host_info, sizeof(h));
    auto asd = [](unsigned long long b) {
        double d;
        memcpy(&d, &b, 8);
        return d;
    };
    memset(out, 0, sizeof(*out));
    out->breakdown_step = h.breakdown_step == ~0ull ? -1 : (int64_t)h.breakdown_step;
    out->min_abs_pivot = asd(h.min_abs_pivot);
    out->max_abs_pivot = asd(h.max_abs_pivot);
    const double cmax = asd(h.max_abs_c);
    out->growth = cmax > 0 ? asd(h.max_abs_u) / cmax : 0.0;
    out->refine_iters = h.refine_iters;
    out->krylov_steps = h.krylov_steps;
    for (int i = 0; i <= GENP_MAX_REFINE; ++i) out->bwd_err[i] = h.bwd_err[i];
    out->status = out->breakdown_step >= 0 ? GENP_ERR_BREAKDOWN : h.refine_status;
    return GENP_OK;
}

}  // extern "C"
