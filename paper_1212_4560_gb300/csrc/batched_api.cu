// batched_api.cu -- plan, autotuner and entry points of the batched solves.
//
// The plan lays the caller's pools out back to back in the caller's order,
// sorts the work queue by size (largest first: longest-processing-time
// scheduling over the persistent CTAs), picks the CTA GEMM tile per size
// class (optionally timed on this GPU) and allocates every workspace, so a
// run only enqueues the multiplier draw, a memset and the batched kernel
// (plus the escalation kernel when the plan has it).
#include "genp_internal.cuh"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <vector>

using namespace genp;

struct genp_batched_plan {
    int64_t count = 0, nrhs = 0;
    genp_mult_kind kind = GENP_MULT_GAUSSIAN;
    genp_prec a_prec = GENP_FP64;
    int max_iter = 0;
    double tol = 0.0;
    int grid = 0, esc_grid = 0, nmax = 0;
    std::vector<int64_t> n, mat_off, vec_off;
    int tile_class[3] = {64, 64, 128};   // CTA GEMM tile for n <= 64, n <= 256, n <= 1024
    BatchDesc *desc = nullptr;
    int *counter = nullptr;              // [0] main queue, [1] escalation queue
    BatchStatus *stat = nullptr;
    float *C = nullptr, *G = nullptr, *g = nullptr;
    float *scratch = nullptr;            // per-CTA scratch, grid x batched_scratch_stride()
    double *R = nullptr;                 // escalation residuals, FP64, vector-pool layout
    double *L = nullptr;                 // adjoint Lambda, FP64, vector-pool layout
    double *scratch64 = nullptr;         // escalation scratch, esc_grid x batched_escalate_stride()
    unsigned long long *prof = nullptr;  // phase profile, grid x kBatchedPhases (when enabled)
    bool have_factors = false;
};

namespace {

int size_class(int64_t n) { return n <= 64 ? 0 : (n <= 256 ? 1 : 2); }

std::mutex g_tune_mu;
std::map<std::string, int> g_tune;   // per-process tuning results

std::string tune_key(int cls, int64_t nrhs, genp_mult_kind kind, genp_prec a_prec) {
    char b[128];
    snprintf(b, sizeof b, "sm_103a/tile/class%d/rhs%lld/kind%d/a%d", cls, (long long)nrhs, (int)kind, (int)a_prec);
    return b;
}

void cache_load() {
    const char *path = getenv("GENP_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char key[128];
    int nb;
    while (fscanf(f, "%127s %d", key, &nb) == 2) g_tune[key] = nb;
    fclose(f);
}

void cache_store() {
    const char *path = getenv("GENP_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "w");
    if (!f) return;
    for (auto &kv : g_tune) fprintf(f, "%s %d\n", kv.first.c_str(), kv.second);
    fclose(f);
}

void free_plan(genp_batched_plan *P) {
    cudaFree(P->desc);
    cudaFree(P->counter);
    cudaFree(P->stat);
    cudaFree(P->C);
    cudaFree(P->G);
    cudaFree(P->g);
    cudaFree(P->scratch);
    cudaFree(P->R);
    cudaFree(P->L);
    cudaFree(P->scratch64);
    cudaFree(P->prof);
    delete P;
}

template <typename T>
bool dmalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    if (cudaMalloc((void **)p, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    return true;
}

// Upload descriptors for the work queue (largest first) with the current block sizes.
cudaError_t upload_desc(genp_batched_plan *P, cudaStream_t s) {
    std::vector<int64_t> order(P->count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return P->n[a] > P->n[b]; });
    std::vector<BatchDesc> h(P->count);
    int64_t goff = 0;
    std::vector<int64_t> g_off(P->count);
    for (int64_t i = 0; i < P->count; ++i) {
        g_off[i] = goff;
        goff += P->n[i];
    }
    for (int64_t q = 0; q < P->count; ++q) {
        const int64_t i = order[q];
        BatchDesc d{};
        d.n = P->n[i];
        d.mat_off = P->mat_off[i];
        d.vec_off = P->vec_off[i];
        d.g_off = g_off[i];
        d.sid = i;
        d.nb = P->tile_class[size_class(P->n[i])];
        h[q] = d;
    }
    cudaError_t e = cudaMemcpyAsync(P->desc, h.data(), h.size() * sizeof(BatchDesc), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

BatchedArgs run_args(genp_batched_plan *P, const void *A, bool a64, const double *B, double *X) {
    BatchedArgs a{};
    a.desc = P->desc;
    a.count = (int)P->count;
    a.counter = P->counter;
    a.A = A;
    a.a64 = a64 ? 1 : 0;
    a.B = B;
    a.X = X;
    a.C = P->C;
    a.G = P->G;
    a.g = P->g;
    a.scratch = P->scratch;
    a.nmax = P->nmax;
    a.nr = (int)P->nrhs;
    a.circ = P->kind == GENP_MULT_CIRCULANT ? 1 : 0;
    a.max_iter = P->max_iter;
    a.tol = P->tol;
    a.stat = P->stat;
    a.prof = P->prof;
    return a;
}

// Times the candidate tiles of one size class on a synthetic batch of
// systems of that class's median order (A = the class's drawn multipliers,
// which are as good a matrix as any for timing; no refinement).
int tune_class(genp_batched_plan *P, int cls, cudaStream_t s) {
    static const int cand[2] = {64, 128};
    std::vector<int64_t> ns;
    for (int64_t v : P->n)
        if (size_class(v) == cls) ns.push_back(v);
    if (ns.empty() || cls == 0) return P->tile_class[cls];
    std::sort(ns.begin(), ns.end());
    const int64_t nm = ns[ns.size() / 2];
    const int reps = (int)std::min<int64_t>(2 * (int64_t)P->grid, std::max<int64_t>((int64_t)ns.size(), 152));
    genp_batched_plan T;
    T.count = reps;
    T.nrhs = P->nrhs;
    T.kind = P->kind;
    T.a_prec = GENP_FP32;
    T.grid = P->grid;
    T.nmax = P->nmax;
    T.n.assign(reps, nm);
    for (int64_t i = 0; i <= reps; ++i) {
        T.mat_off.push_back(i * nm * nm);
        T.vec_off.push_back(i * nm * P->nrhs);
    }
    const size_t mats = (size_t)reps * nm * nm, vecs = (size_t)reps * nm * P->nrhs;
    float *A = nullptr;
    double *B = nullptr, *X = nullptr;
    int best = P->tile_class[cls];
    auto release = [&]() {
        cudaFree(A); cudaFree(B); cudaFree(X);
        cudaFree(T.desc); cudaFree(T.counter); cudaFree(T.stat); cudaFree(T.C); cudaFree(T.G); cudaFree(T.g);
        T.desc = nullptr;
        T.counter = nullptr;
        T.stat = nullptr;
        T.C = T.G = T.g = nullptr;
    };
    if (!dmalloc(&A, mats) || !dmalloc(&B, vecs) || !dmalloc(&X, vecs) || !dmalloc(&T.desc, reps) ||
        !dmalloc(&T.counter, 2) || !dmalloc(&T.stat, reps) || !dmalloc(&T.C, mats) || !dmalloc(&T.G, mats) ||
        !dmalloc(&T.g, (size_t)reps * nm)) {
        release();
        return best;
    }
    T.scratch = P->scratch;   // the plan's own per-CTA scratch (same grid, nmax and nrhs)
    T.prof = nullptr;
    T.max_iter = 0;
    T.tol = 0.0;
    cudaMemsetAsync(B, 0, vecs * sizeof(double), s);
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int c = 0; c < 2; ++c) {
        const int ts = cand[c];
        for (int k = 0; k < 3; ++k) T.tile_class[k] = ts;
        if (upload_desc(&T, s) != cudaSuccess) break;
        launch_batch_draw(T.desc, (int)reps, 12345, false, A, T.g, s);
        float ms = 0.f;
        for (int r = 0; r < 2; ++r) {
            cudaEventRecord(e0, s);
            launch_batched(run_args(&T, A, false, B, X), T.grid, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
        }
        if (cudaGetLastError() == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = ts;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    T.scratch = nullptr;
    release();
    return best;
}

}  // namespace

extern "C" {

genp_status genp_batched_plan_create(int64_t count, const int64_t *n, int64_t nrhs, genp_mult_kind kind,
                                     genp_prec a_prec, int max_iter, double tol, int flags, void *cuda_stream,
                                     genp_batched_plan **out) {
    const bool autotune = (flags & GENP_BATCH_AUTOTUNE) != 0, escalate = (flags & GENP_BATCH_FP64_ESCALATION) != 0;
    if (!out) return GENP_ERR_ARG;
    *out = nullptr;
    if (count < 1 || count > (1ll << 30) || !n || nrhs < 1 || nrhs > 16) return GENP_ERR_ARG;
    if (kind != GENP_MULT_GAUSSIAN && kind != GENP_MULT_CIRCULANT) return GENP_ERR_ARG;
    if (a_prec != GENP_FP64 && a_prec != GENP_FP32) return GENP_ERR_ARG;
    if (max_iter < 0 || max_iter > GENP_MAX_REFINE || !(tol >= 0.0)) return GENP_ERR_ARG;
    for (int64_t i = 0; i < count; ++i)
        if (n[i] < 1 || n[i] > 1024) return GENP_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    genp_batched_plan *P = new (std::nothrow) genp_batched_plan();
    if (!P) return GENP_ERR_NOMEM;
    P->count = count;
    P->nrhs = nrhs;
    P->kind = kind;
    P->a_prec = a_prec;
    P->max_iter = max_iter;
    P->tol = tol;
    P->n.assign(n, n + count);
    int64_t mo = 0, vo = 0;
    for (int64_t i = 0; i < count; ++i) {
        P->mat_off.push_back(mo);
        P->vec_off.push_back(vo);
        mo += n[i] * n[i];
        vo += n[i] * nrhs;
    }
    P->mat_off.push_back(mo);
    P->vec_off.push_back(vo);
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    P->nmax = (int)*std::max_element(n, n + count);
    const int per_sm = batched_blocks_per_sm((int)nrhs, P->nmax);
    if (per_sm < 1) {
        cudaGetLastError();
        free_plan(P);
        return GENP_ERR_CUDA;
    }
    // one persistent CTA per resident slot, no more than there are systems
    P->grid = (int)std::min<int64_t>((int64_t)sms * per_sm, count);
    P->esc_grid = escalate ? (int)std::min<int64_t>((int64_t)sms * batched_escalate_blocks_per_sm(), count) : 0;
    const bool circ = kind == GENP_MULT_CIRCULANT;
    if (!dmalloc(&P->desc, count) || !dmalloc(&P->counter, 2) || !dmalloc(&P->stat, count) ||
        !dmalloc(&P->C, mo) || (!circ && !dmalloc(&P->G, mo)) || (circ && !dmalloc(&P->g, vo / nrhs)) ||
        !dmalloc(&P->scratch, (size_t)P->grid * batched_scratch_stride((int)nrhs, P->nmax)) ||
        !dmalloc(&P->L, vo) || (escalate && !dmalloc(&P->R, vo)) ||
        (escalate && !dmalloc(&P->scratch64, (size_t)P->esc_grid * batched_escalate_stride()))) {
        free_plan(P);
        return GENP_ERR_NOMEM;
    }
    if (autotune) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        static bool loaded = false;
        if (!loaded) {
            cache_load();
            loaded = true;
        }
        bool changed = false;
        for (int cls = 0; cls < 3; ++cls) {
            const std::string key = tune_key(cls, nrhs, kind, a_prec);
            auto it = g_tune.find(key);
            if (it != g_tune.end()) {
                P->tile_class[cls] = it->second;
                continue;
            }
            bool present = false;
            for (int64_t v : P->n) present = present || size_class(v) == cls;
            if (!present) continue;
            P->tile_class[cls] = tune_class(P, cls, s);
            g_tune[key] = P->tile_class[cls];
            changed = true;
        }
        if (changed) cache_store();
    }
    if (upload_desc(P, s) != cudaSuccess) {
        cudaGetLastError();
        free_plan(P);
        return GENP_ERR_CUDA;
    }
    *out = P;
    return GENP_OK;
}

genp_status genp_batched_layout(const genp_batched_plan *P, int64_t *mat_offsets, int64_t *vec_offsets) {
    if (!P) return GENP_ERR_ARG;
    if (mat_offsets) memcpy(mat_offsets, P->mat_off.data(), P->mat_off.size() * sizeof(int64_t));
    if (vec_offsets) memcpy(vec_offsets, P->vec_off.data(), P->vec_off.size() * sizeof(int64_t));
    return GENP_OK;
}

int genp_batched_block_size(const genp_batched_plan *P, int64_t n) {
    if (!P || n < 1) return 0;
    return P->tile_class[size_class(n)];
}

genp_status genp_batched_run(genp_batched_plan *P, uint64_t seed, const void *A_pool, const double *B_pool,
                             double *X_pool, void *cuda_stream) {
    if (!P || !A_pool || !B_pool || !X_pool) return GENP_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const bool circ = P->kind == GENP_MULT_CIRCULANT;
    const bool a64 = P->a_prec == GENP_FP64;
    if (launch_batch_draw(P->desc, (int)P->count, seed, circ, P->G, P->g, s) != cudaSuccess ||
        launch_batched(run_args(P, A_pool, a64, B_pool, X_pool), P->grid, s) != cudaSuccess) {
        cudaGetLastError();
        return GENP_ERR_CUDA;
    }
    if (P->scratch64 && P->max_iter > 0) {
        if (cudaMemsetAsync(P->counter + 1, 0, sizeof(int), s) != cudaSuccess ||
            launch_batched_escalate(P->desc, (int)P->count, P->counter + 1, A_pool, a64, B_pool, X_pool, P->G, P->g,
                                    P->R, P->scratch64, (int)P->nrhs, circ, P->max_iter, P->tol, P->stat,
                                    P->esc_grid, s) != cudaSuccess) {
            cudaGetLastError();
            return GENP_ERR_CUDA;
        }
    }
    P->have_factors = true;
    return GENP_OK;
}

genp_status genp_batched_adjoint(genp_batched_plan *P, const void *A_pool, const double *gX_pool, const double *X_pool,
                                 float *dA_pool, double *dB_pool, void *cuda_stream) {
    if (!P || !A_pool || !gX_pool || !P->have_factors) return GENP_ERR_ARG;
    if (dA_pool && !X_pool) return GENP_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    BatchedArgs a = run_args(P, A_pool, P->a_prec == GENP_FP64, nullptr, const_cast<double *>(X_pool));
    a.gX = gX_pool;
    a.L = P->L;
    a.dB = dB_pool;
    a.dA = dA_pool;
    if (launch_batched_adjoint(a, P->grid, s) != cudaSuccess) {
        cudaGetLastError();
        return GENP_ERR_CUDA;
    }
    return GENP_OK;
}

genp_status genp_batched_status(const genp_batched_plan *P, int32_t *status, int32_t *iters, double *eta0,
                                double *eta, double *growth, int32_t *escalated, int32_t *krylov,
                                void *cuda_stream) {
    if (!P) return GENP_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    std::vector<BatchStatus> h(P->count);
    std::vector<BatchDesc> d(P->count);
    if (cudaMemcpyAsync(h.data(), P->stat, h.size() * sizeof(BatchStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(d.data(), P->desc, d.size() * sizeof(BatchDesc), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return GENP_ERR_CUDA;
    }
    // the status array is in work-queue order; report in the caller's order
    for (int64_t q = 0; q < P->count; ++q) {
        const int64_t i = d[q].sid;
        if (status) status[i] = h[q].status;
        if (iters) iters[i] = h[q].refine_iters;
        if (eta0) eta0[i] = h[q].eta0;
        if (eta) eta[i] = h[q].eta;
        if (growth) growth[i] = h[q].max_abs_c > 0 ? (double)h[q].max_abs_u / h[q].max_abs_c : 0.0;
        if (escalated) escalated[i] = h[q].escalated;
        if (krylov) krylov[i] = h[q].krylov_steps;
    }
    return GENP_OK;
}

genp_status genp_batched_multipliers(const genp_batched_plan *P, float *G_pool, float *g_pool, void *cuda_stream) {
    if (!P) return GENP_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (G_pool) {
        if (!P->G) return GENP_ERR_ARG;
        if (cudaMemcpyAsync(G_pool, P->G, P->mat_off.back() * sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return GENP_ERR_CUDA;
    }
    if (g_pool) {
        if (!P->g) return GENP_ERR_ARG;
        if (cudaMemcpyAsync(g_pool, P->g, P->vec_off.back() / P->nrhs * sizeof(float), cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
            return GENP_ERR_CUDA;
    }
    return GENP_OK;
}

genp_status genp_batched_profile(genp_batched_plan *P, int enable) {
    if (!P) return GENP_ERR_ARG;
    if (!enable) {
        cudaFree(P->prof);
        P->prof = nullptr;
        return GENP_OK;
    }
    if (!P->prof) {
        if (!dmalloc(&P->prof, (size_t)P->grid * kBatchedPhases)) return GENP_ERR_NOMEM;
        if (cudaMemset(P->prof, 0, (size_t)P->grid * kBatchedPhases * sizeof(unsigned long long)) != cudaSuccess)
            return GENP_ERR_CUDA;
    }
    return GENP_OK;
}

genp_status genp_batched_profile_read(const genp_batched_plan *P, double *cycles, void *cuda_stream) {
    if (!P || !P->prof || !cycles) return GENP_ERR_ARG;
    std::vector<unsigned long long> h((size_t)P->grid * kBatchedPhases);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (cudaMemcpyAsync(h.data(), P->prof, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return GENP_ERR_CUDA;
    }
    for (int p = 0; p < kBatchedPhases; ++p) {
        double t = 0.0;
        for (int b = 0; b < P->grid; ++b) t += (double)h[(size_t)b * kBatchedPhases + p];
        cycles[p] = t;
    }
    return GENP_OK;
}

void genp_batched_plan_destroy(genp_batched_plan *P) {
    if (P) free_plan(P);
}

}  // extern "C"
