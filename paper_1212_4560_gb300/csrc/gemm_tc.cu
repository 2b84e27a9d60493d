// gemm_tc.cu -- tensor-core GEMMs on sm_103a (tcgen05 + TMA + TMEM).  First
// the BF16 one:
//   D (fp32, row-major) = alpha * A * B^T + beta * Cin
// with A (m x K) and B (n x K) BF16, both K-major (row-major with K
// contiguous), FP32 accumulation in tensor memory.  It serves the mixed
// precision path of the method: the Schur-complement update of block
// Gaussian elimination (Thm. 2.2's block form) with BF16 (or split-BF16)
// operands and an FP32 master trailing matrix, and the product C = A G of
// Thm. 4.1 with G on the BF16 grid.
//
// One 128 x 128 output tile per CTA (grid = tiles), 128 threads:
//   warp 0, one lane: TMA producer, 3-stage ring of 128 x 64 A and B tiles
//                     (128-byte rows, 128B swizzle) in shared memory;
//   warp 1: allocates 128 TMEM columns; one lane issues tcgen05.mma
//           (M = 128, N = 128, K = 16 per instruction) and commits each
//           stage back to the producer;
//   all 4 warps: epilogue, warp w reads TMEM lanes 32w..32w+31 (its rows).
// Two CTAs fit per SM (96 KiB of stages each), so one CTA's epilogue
// overlaps the other's main loop.  Every mbarrier wait is bounded: after
// ~2 s it sets g_tc_timeout, stops issuing, drains what it issued (bounded)
// and frees its TMEM, so a broken pipeline returns an error, never a hang.
#include "genp_internal.cuh"

#include <cuda.h>
#include <utility>
#include <vector>
#include <cudaTypedefs.h>

#include "dfloat.cuh"
#include "sliced.cuh"

__device__ int g_tc_timeout;

namespace genp {
namespace {

constexpr int BM = 128, BN = 128, BK = 64, UMMA_K = 16, STAGES = 3;
constexpr uint32_t A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
constexpr uint32_t TMEM_COLS = 128;
constexpr long long kTimeout = 4000000000LL;  // clock64 ticks (~2 s at 2 GHz)

struct Ctl {
    unsigned long long full[STAGES];
    unsigned long long empty[STAGES];
    unsigned long long accum;
    uint32_t tmem;
    int abort;
    int issued;
};
constexpr size_t kSmem = 1024 + STAGES * (A_BYTES + B_BYTES) + sizeof(Ctl);
// Epilogue tile row stride in floats: 16-byte aligned rows whose bank offset
// (132 mod 32 = 4) makes the per-row float4 writes and the row reads
// conflict-free.
constexpr int kTileLd = BN + 4;
static_assert(BM * kTileLd * 4 <= STAGES * (A_BYTES + B_BYTES), "epilogue tile fits in the stage buffers");

__device__ __forceinline__ uint32_t sa(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned long long *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(sa(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait; false on timeout or when another thread has aborted.
__device__ bool mbar_wait(unsigned long long *b, uint32_t parity, volatile int *abort) {
    const long long t0 = clock64();
    while (!mbar_try(b, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > kTimeout) return false;
    }
    return true;
}
__device__ __forceinline__ void tma_2d(void *dst, const CUtensorMap *map, unsigned long long *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(sa(dst)), "l"((uint64_t)map), "r"(sa(bar)), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte rows with the
// 128B swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);   // start address / 16
    d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                   // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                   // 128B swizzle
    return d;
}
// Instruction descriptor, kind::f16: D F32, A and B BF16, both K-major, M x N.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void commit(unsigned long long *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sa(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(b)) : "memory");
}
// barrier among the 128 epilogue threads only
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Instruction descriptor, kind::f8f6f4: D F32, A and B E4M3 (format 0), both K-major, M x N.
constexpr uint32_t kIdescE4M3 = (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_e4m3(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(kIdescE4M3), "r"(acc)
        : "memory");
}

// Q8: e4m3 operands (kind::f8f6f4, 128 per 128-byte k-tile row, K = 32 per
// MMA) with K <= 128, so that one scale product scA[tm] scB[tn] covers the
// whole tile and joins alpha in the epilogue (the Schur updates of
// GENP_FP8_E4M3: K = nb).
template <bool Q8>
__global__ void __launch_bounds__(128, 2)
k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int m, int n, int K,
          float alpha, float beta, const float *Cin, int64_t ldci, float *D, int64_t ldd, int vec, const int *skip,
          const float *scA, const float *scB) {
    if (skip && *skip) return;
    extern __shared__ unsigned char smraw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = base;
    unsigned char *sB = base + STAGES * A_BYTES;
    Ctl *ctl = (Ctl *)(sB + STAGES * B_BYTES);
    volatile int *abort = &ctl->abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    constexpr int kStep = Q8 ? 2 * BK : BK;   // elements per 128-byte k-tile row
    const int nk = (K + kStep - 1) / kStep;
    if (Q8) alpha *= scA[blockIdx.y] * scB[blockIdx.x];

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&ctl->full[s], 1);
            mbar_init(&ctl->empty[s], 1);
        }
        mbar_init(&ctl->accum, 1);
        ctl->abort = 0;
        ctl->issued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(&ctl->tmem)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = ctl->tmem;
    // the tile's rows of Cin into L2 while the main loop runs (the epilogue's
    // read-modify-write of C is most of a short-K product's traffic)
    if (beta != 0.0f && m0 + (int)threadIdx.x < m && n0 < n) {
        const char *rp = reinterpret_cast<const char *>(Cin + (int64_t)(m0 + threadIdx.x) * ldci + n0);
        const int bytes = (n - n0 < BN ? n - n0 : BN) * (int)sizeof(float);
        for (int b = 0; b < bytes; b += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(rp + b));
    }

    if (warp == 0 && lane == 0) {
        // producer
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % STAGES;
            const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
            if (kt >= STAGES && !mbar_wait(&ctl->empty[s], ph ^ 1u, abort)) {
                *abort = 1;
                break;
            }
            mbar_expect_tx(&ctl->full[s], A_BYTES + B_BYTES);
            tma_2d(sA + s * A_BYTES, &tmA, &ctl->full[s], kt * kStep, m0);
            tma_2d(sB + s * B_BYTES, &tmB, &ctl->full[s], kt * kStep, n0);
            ctl->issued = kt + 1;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        bool ok = true;
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % STAGES;
            const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
            if (!mbar_wait(&ctl->full[s], ph, abort)) {
                *abort = 1;
                ok = false;
                break;
            }
            fence_after();
            const uint64_t ad = sdesc(sa(sA + s * A_BYTES)), bd = sdesc(sa(sB + s * B_BYTES));
#pragma unroll
            for (int k = 0; k < BK / UMMA_K; ++k) {  // +32 bytes along K inside the swizzle atom
                if (Q8)
                    mma_e4m3(tmem, ad + (uint64_t)(k * 2), bd + (uint64_t)(k * 2), (kt > 0 || k > 0) ? 1u : 0u);
                else
                    mma(tmem, ad + (uint64_t)(k * 2), bd + (uint64_t)(k * 2), (kt > 0 || k > 0) ? 1u : 0u);
            }
            commit(&ctl->empty[s]);
        }
        if (ok) commit(&ctl->accum);
    }
    __syncwarp();

    // epilogue: TMEM -> registers -> shared memory (the stage buffers are free
    // once the accumulator is complete) -> coalesced rows of D
    bool ready = mbar_wait(&ctl->accum, 0, abort);
    if (!ready) *abort = 1;
    fence_after();
    ready = __syncthreads_and(ready) != 0;
    float *tile = reinterpret_cast<float *>(base);  // BM x kTileLd floats
    if (ready) {
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        float4 *trow = reinterpret_cast<float4 *>(tile + (warp * 32 + lane) * kTileLd);
#pragma unroll 1
        for (int c = 0; c < BN / 32; ++c) {
            uint32_t r[32];
            tmem_ld32(lane_addr + (uint32_t)(c * 32), r);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                trow[c * 8 + q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                              __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
        }
    }
    __syncthreads();
    if (ready) {
        const int col = n0 + lane * 4;
        for (int rr = warp; rr < BM; rr += 4) {
            const int row = m0 + rr;
            if (row >= m) break;
            const float4 a = *reinterpret_cast<const float4 *>(tile + rr * kTileLd + lane * 4);
            float *drow = D + (int64_t)row * ldd;
            if (vec && col + 3 < n) {
                float4 v = make_float4(alpha * a.x, alpha * a.y, alpha * a.z, alpha * a.w);
                if (beta != 0.0f) {
                    const float4 cv = *reinterpret_cast<const float4 *>(Cin + (int64_t)row * ldci + col);
                    v.x = fmaf(beta, cv.x, v.x);
                    v.y = fmaf(beta, cv.y, v.y);
                    v.z = fmaf(beta, cv.z, v.z);
                    v.w = fmaf(beta, cv.w, v.w);
                }
                *reinterpret_cast<float4 *>(drow + col) = v;
            } else {
                const float av[4] = {a.x, a.y, a.z, a.w};
                for (int e = 0; e < 4; ++e) {
                    if (col + e >= n) break;
                    float v = alpha * av[e];
                    if (beta != 0.0f) v = fmaf(beta, Cin[(int64_t)row * ldci + col + e], v);
                    drow[col + e] = v;
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (ctl->abort) {
        if (threadIdx.x == 0) {
            atomicExch(&g_tc_timeout, 1);
            // drain the copies this CTA issued before freeing its shared memory
            const int issued = ctl->issued;
            int dummy = 0;
            for (int kt = (issued > STAGES ? issued - STAGES : 0); kt < issued; ++kt)
                mbar_wait(&ctl->full[kt % STAGES], (uint32_t)(kt / STAGES) & 1u, (volatile int *)&dummy);
        }
        // outstanding MMAs signal accum (or empty); wait for it (bounded) before freeing TMEM
        if (threadIdx.x == 32) {
            int dummy = 0;
            mbar_wait(&ctl->accum, 0, (volatile int *)&dummy);
        }
        __syncthreads();
    }
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2-D BF16 map of a rows x K row-major matrix, box BK x box_rows, 128B swizzle.
bool make_map(CUtensorMap *map, const void *ptr, int64_t rows, int64_t K, int64_t ld, int box_rows) {
    auto fn = encoder();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ---------------------------------------------------------------------------
// E4M3 product with a power-of-two scale per 128 x 128 operand tile:
//   D = alpha * sum_kt scA[tm][kt] scB[tn][kt] (A_kt B_kt^T) + beta * Cin
// A (m x K) and B^T (n x K) hold e4m3 codes, K-major; tile (tm, kt) of A is
// rows 128 tm .. and columns 128 kt .., its scale scA[tm * nkt + kt]
// (nkt = ceil(K / 128)); likewise scB for B^T.  Each k-tile (128 e4m3 = one
// 128-byte swizzle row) is four K = 32 tcgen05 kind::f8f6f4 MMAs.  A run of
// consecutive k-tiles with the same scale product sc (exact powers of two,
// compared exactly) accumulates in one TMEM accumulator, since
// sum sc P_kt = sc sum P_kt; at the end of the run the epilogue warps read
// it and add it, times sc, into FP32 registers while the MMAs of the next
// run fill the other accumulator.  Tiles of similar magnitude share their
// scales, so a row of tiles is mostly one run.
//   warps 0-7: promotion and the final write (warp w: TMEM lanes 32 (w % 4)
//              .. = its rows, columns 64 (w / 4) .. = its half; two warps per
//              scheduler keep the promotion ahead of the MMAs);
//   warp 8, one lane: TMA producer, six stages of A and B tiles (192 KiB:
//              the loads in flight cover the latency at 32 KiB per k-tile);
//   warp 9, one lane: MMA issue.
// One CTA per SM; every wait is bounded.
// ---------------------------------------------------------------------------
constexpr int QBK = 128, Q_STAGES = 6, kQEpiWarps = 8, kQThreads = 32 * (kQEpiWarps + 2);
constexpr int kQProducer = kQEpiWarps, kQMma = kQEpiWarps + 1;   // warp indices
constexpr uint32_t QA_BYTES = BM * QBK, QB_BYTES = BN * QBK;
constexpr uint32_t Q_TMEM = 256;
// barrier among the epilogue warps only
__device__ __forceinline__ void epi_sync_q() { asm volatile("bar.sync 1, %0;" ::"n"(32 * kQEpiWarps) : "memory"); }
struct QCtl {
    unsigned long long full[Q_STAGES];
    unsigned long long empty[Q_STAGES];
    unsigned long long afull[2];     // accumulator b holds a finished k-tile
    unsigned long long aempty[2];    // the epilogue has read accumulator b (4 arrivals)
    unsigned long long drain;
    uint32_t tmem;
    int abort;
    int issued;
};
constexpr int kQMaxKt = 2048;     // k-tiles whose scale products the CTA keeps (K <= 262144)
constexpr size_t kQSmem = 1024 + Q_STAGES * (QA_BYTES + QB_BYTES) + sizeof(QCtl) + kQMaxKt * sizeof(float);
static_assert(kQSmem <= 227 * 1024, "shared memory");
static_assert(BM * kTileLd * 4 <= Q_STAGES * (QA_BYTES + QB_BYTES), "output tile fits in the stage buffers");

__global__ void __launch_bounds__(kQThreads, 1)
k_tc_e4m3(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int m, int n, int K,
          float alpha, const float *scA, const float *scB, float beta, const float *Cin, int64_t ldci, float *D,
          int64_t ldd, int vec) {
    extern __shared__ unsigned char smraw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = base;
    unsigned char *sB = base + Q_STAGES * QA_BYTES;
    QCtl *ctl = (QCtl *)(sB + Q_STAGES * QB_BYTES);
    float *s_sc = reinterpret_cast<float *>(ctl + 1);   // scale product of each k-tile
    volatile int *abort = &ctl->abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tm = blockIdx.y, tn = blockIdx.x;
    const int m0 = tm * BM, n0 = tn * BN;
    const int nkt = (K + QBK - 1) / QBK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < Q_STAGES; ++s) {
            mbar_init(&ctl->full[s], 1);
            mbar_init(&ctl->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&ctl->afull[b], 1);
            mbar_init(&ctl->aempty[b], kQEpiWarps);
        }
        mbar_init(&ctl->drain, 1);
        ctl->abort = 0;
        ctl->issued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kQMma) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(&ctl->tmem)),
                     "r"(Q_TMEM)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int kt = threadIdx.x; kt < nkt; kt += blockDim.x)
        s_sc[kt] = scA[(int64_t)tm * nkt + kt] * scB[(int64_t)tn * nkt + kt];
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = ctl->tmem;

    if (warp == kQProducer) {
        if (lane == 0) {
            for (int kt = 0; kt < nkt; ++kt) {
                const int s = kt % Q_STAGES;
                if (kt >= Q_STAGES && !mbar_wait(&ctl->empty[s], (uint32_t)((kt / Q_STAGES) & 1) ^ 1u, abort)) {
                    *abort = 1;
                    break;
                }
                mbar_expect_tx(&ctl->full[s], QA_BYTES + QB_BYTES);
                tma_2d(sA + s * QA_BYTES, &tmA, &ctl->full[s], kt * QBK, m0);
                tma_2d(sB + s * QB_BYTES, &tmB, &ctl->full[s], kt * QBK, n0);
                ctl->issued = kt + 1;
            }
        }
        __syncwarp();
    } else if (warp == kQMma) {
        if (lane == 0) {
            int g = -1, b = 0;   // run index, its accumulator
            for (int kt = 0; kt < nkt; ++kt) {
                const int s = kt % Q_STAGES;
                const float sc = s_sc[kt];
                const bool start = kt == 0 || s_sc[kt - 1] != sc;
                const bool last = kt + 1 == nkt || s_sc[kt + 1] != sc;
                if (start) {
                    // accumulator b was last filled by run g - 2
                    ++g;
                    b = g & 1;
                    if (g >= 2 && !mbar_wait(&ctl->aempty[b], (uint32_t)(((g - 2) >> 1) & 1), abort)) {
                        *abort = 1;
                        break;
                    }
                }
                if (!mbar_wait(&ctl->full[s], (uint32_t)((kt / Q_STAGES) & 1), abort)) {
                    *abort = 1;
                    break;
                }
                fence_after();
                const uint64_t ad = sdesc(sa(sA + s * QA_BYTES)), bd = sdesc(sa(sB + s * QB_BYTES));
#pragma unroll
                for (int k = 0; k < QBK / 32; ++k)   // K = 32 e4m3 (32 bytes) per MMA
                    mma_e4m3(tmem + (uint32_t)(b * BN), ad + (uint64_t)(k * 2), bd + (uint64_t)(k * 2),
                             (start && k == 0) ? 0u : 1u);
                commit(&ctl->empty[s]);
                if (last) commit(&ctl->afull[b]);
            }
        }
        __syncwarp();
    } else {
        // promotion: acc += scA scB P_kt.  Epilogue warp w reads TMEM lanes
        // 32 (w % 4) .. (its rows) and columns 64 (w / 4) .. (its half).
        constexpr int HALF = BN / 2;
        const int row = (warp & 3) * 32 + lane, h = warp >> 2;
        const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(h * HALF);
        float acc[HALF];
#pragma unroll
        for (int j = 0; j < HALF; ++j) acc[j] = 0.0f;
        bool ok = true;
        for (int kt = 0, g = 0; kt < nkt; ++g) {
            const int b = g & 1;
            const float sc = s_sc[kt];
            int e = kt + 1;                    // the run is k-tiles kt .. e - 1
            while (e < nkt && s_sc[e] == sc) ++e;
            kt = e;
            if (!mbar_wait(&ctl->afull[b], (uint32_t)((g >> 1) & 1), abort)) {
                *abort = 1;
                ok = false;
                break;
            }
            fence_after();
#pragma unroll
            for (int c = 0; c < HALF / 32; ++c) {
                uint32_t q[32];
                tmem_ld32(lane_addr + (uint32_t)(b * BN + c * 32), q);
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[c * 32 + j] = fmaf(sc, __uint_as_float(q[j]), acc[c * 32 + j]);
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl->aempty[b]);
        }
        // every k-tile is consumed, so the stage buffers are free: rows through
        // shared memory, then coalesced rows of D
        epi_sync_q();
        ok = ok && !*abort;
        float *tile = reinterpret_cast<float *>(base);   // BM x kTileLd
        if (ok) {
            float4 *trow = reinterpret_cast<float4 *>(tile + row * kTileLd + h * HALF);
#pragma unroll
            for (int q = 0; q < HALF / 4; ++q)
                trow[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
        }
        epi_sync_q();
        if (ok) {
            const int col = n0 + lane * 4;
            for (int rr = warp; rr < BM; rr += kQEpiWarps) {
                const int row = m0 + rr;
                if (row >= m) break;
                const float4 a = *reinterpret_cast<const float4 *>(tile + rr * kTileLd + lane * 4);
                float *drow = D + (int64_t)row * ldd;
                if (vec && col + 3 < n) {
                    float4 v = make_float4(alpha * a.x, alpha * a.y, alpha * a.z, alpha * a.w);
                    if (beta != 0.0f) {
                        const float4 cv = *reinterpret_cast<const float4 *>(Cin + (int64_t)row * ldci + col);
                        v.x = fmaf(beta, cv.x, v.x);
                        v.y = fmaf(beta, cv.y, v.y);
                        v.z = fmaf(beta, cv.z, v.z);
                        v.w = fmaf(beta, cv.w, v.w);
                    }
                    *reinterpret_cast<float4 *>(drow + col) = v;
                } else {
                    const float av[4] = {a.x, a.y, a.z, a.w};
                    for (int e = 0; e < 4; ++e) {
                        if (col + e >= n) break;
                        float v = alpha * av[e];
                        if (beta != 0.0f) v = fmaf(beta, Cin[(int64_t)row * ldci + col + e], v);
                        drow[col + e] = v;
                    }
                }
            }
        }
    }

    fence_before();
    __syncthreads();
    if (ctl->abort) {
        if (threadIdx.x == 32 * kQProducer) {
            atomicExch(&g_tc_timeout, 1);
            int dummy = 0;
            const int issued = ctl->issued;
            for (int kt = (issued > Q_STAGES ? issued - Q_STAGES : 0); kt < issued; ++kt)
                mbar_wait(&ctl->full[kt % Q_STAGES], (uint32_t)((kt / Q_STAGES) & 1), (volatile int *)&dummy);
        }
        if (threadIdx.x == 32 * kQMma) {     // the MMA thread: wait for its MMAs still in flight
            int dummy = 0;
            commit(&ctl->drain);
            mbar_wait(&ctl->drain, 0, (volatile int *)&dummy);
        }
        __syncthreads();
    }
    if (warp == kQMma)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Q_TMEM) : "memory");
}

// 2-D map of a rows x K matrix of bytes (e4m3 codes), box 128 x 128, 128B swizzle.
bool make_map_u8(CUtensorMap *map, const void *ptr, int64_t rows, int64_t K, int64_t ld) {
    auto fn = encoder();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld};
    cuuint32_t box[2] = {(cuuint32_t)QBK, (cuuint32_t)BM};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ---------------------------------------------------------------------------
// Sliced (FP64-class) product (layout in sliced.cuh).  Digit group g = t + u
// accumulates in TMEM columns [64 (g-2), 64 (g-1)), so one MMA of A's digit t
// against B's digits 1 .. ND+1-t laid side by side along N (N = 64 (ND+1-t),
// cut at 256) lands every product in its group's columns.
//
// Persistent and warp-specialized: one CTA per SM walks 128 x 64 tiles.
// Warp 4 issues TMA (B's ND digit slices of a k-tile in one of two stages,
// A's digit slices through a four-slot ring), warp 5 issues tcgen05.mma,
// warps 0-3 (TMEM lanes 0-127) run the epilogue.  The epilogue reads the
// group accumulators and hands TMEM back (tempty) before it scales the sums
// and adds them into D (half a tile at a time through shared memory, rows
// coalesced), so that work and the next tile's first TMA loads overlap the
// next tile's MMAs.  The groups below the last are integers
// below 2^24 (K <= 512), recombined by a double-float Horner scheme on the
// FP32 pipe; the last group is added with its 2^-7:
//   D[i][j] += alpha 2^{e_i + f_j - 7 ND} (sum_{g<=ND} 2^{7(ND-g)} P_g + 2^-7 P_{ND+1})
// Every wait is bounded (then the CTA aborts, drains its copies, frees TMEM).
// ---------------------------------------------------------------------------
constexpr int SBN = 64, A_SLOTS_MAX = 8;
constexpr uint32_t SA_BYTES = BM * BK * 2;      // one A digit slice of a k-tile
constexpr uint32_t SBD_BYTES = SBN * BK * 2;    // one B digit slice of a k-tile
constexpr uint32_t S_TMEM = 512;
constexpr int kSlicedThreads = 192;             // 4 epilogue warps, producer, MMA
constexpr int kHalfLd = 33;                     // epilogue staging: 128 rows x 32 dfloat, padded
constexpr uint32_t STAGE_BYTES = BM * kHalfLd * 8;
struct SCtl {
    unsigned long long afull[A_SLOTS_MAX];
    unsigned long long aempty[A_SLOTS_MAX];
    unsigned long long bfull[2];
    unsigned long long bempty[2];
    unsigned long long tfull;     // a tile's accumulators are complete
    unsigned long long tempty;    // the epilogue has read them (4 arrivals)
    unsigned long long drain;     // outstanding MMAs, on the abort path
    uint32_t tmem;
    int abort;
    int issued_a, issued_b;
    int epi_go;                   // the epilogue warps' common decision to go on
    float cs[SBN];                // alpha 2^{f_j} of the current tile's columns
};

__device__ __forceinline__ void mma_n(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__host__ __device__ constexpr uint32_t idesc_n(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}
// Bounded wait with a sleep between tries: for warps that wait a long time
// while others on the same scheduler issue TMA and MMA instructions.
__device__ bool mbar_wait_sleep(unsigned long long *b, uint32_t parity, volatile int *abort) {
    const long long t0 = clock64();
    while (!mbar_try(b, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > kTimeout) return false;
        __nanosleep(256);
    }
    return true;
}

// One Horner step on two columns at once: (H, L) <- w (H, L) + p, w a power
// of two, as double-float: TwoSum of w H and p by FMA (w H is exact, so each
// FMA rounds once, as the plain sequence does), the error plus w L, then the
// FastTwoSum renormalisation; ten packed FP32 instructions for two columns.
__device__ __forceinline__ void horner2(float2 &H, float2 &L, float2 p, float2 w) {
    const float2 mw = make_float2(-w.x, -w.y), m1 = make_float2(-1.0f, -1.0f);
    const float2 s = __ffma2_rn(H, w, p);
    const float2 bb = __ffma2_rn(H, mw, s);       // s - w H
    const float2 t1 = __ffma2_rn(bb, m1, s);      // s - bb
    const float2 t2n = __ffma2_rn(H, mw, t1);     // t1 - w H
    const float2 t3 = __ffma2_rn(bb, m1, p);      // p - bb
    float2 e = __ffma2_rn(t2n, m1, t3);           // (w H - t1) + (p - bb)
    e = __ffma2_rn(L, w, e);                      // + w L
    const float2 hn = __fadd2_rn(s, e);
    const float2 u = __ffma2_rn(s, m1, hn);       // hn - s
    H = hn;
    L = __ffma2_rn(u, m1, e);                     // e - u
}

// NDA digits of the A operand, NDB of B (an operand whose entries are exact
// in fewer digits, such as a multiplier on a fixed-point grid, takes fewer
// and goes on the M side, so the wide operand's digits lie along N):
// ND = max(NDA, NDB) groups, and A's digit t meets B's digits
// 0 .. min(NDB, ND - t) - 1 in MMAs of N up to 256 covering
// 64 min(NDB, ND - t) columns, so every kept pair (t + u <= ND - 1, 0-based)
// is formed once: NDA = NDB = 7 gives the 28 pairs of the symmetric product,
// NDA = 2 with NDB = 7 gives 13 (in four MMAs of N = 256, 192, 256, 128 per
// 16-deep step).
template <int NDA, int NDB>
struct SlicedCfg {
    static constexpr int ND = NDA > NDB ? NDA : NDB;
    static constexpr int kPairs = [] {
        int p = 0;
        for (int t = 0; t < NDA; ++t) p += NDB < ND - t ? NDB : ND - t;
        return p;
    }();
    static constexpr uint32_t kBStage = NDB * SBD_BYTES;
    // as deep a ring of A digit slices as the shared memory left by B's two
    // stages and the epilogue's staging allows (the loads take longer than
    // the MMAs of the few slices a four-slot ring keeps in flight)
    static constexpr size_t kFixed = 1024 + 2 * kBStage + STAGE_BYTES + sizeof(SCtl);
    static constexpr int kASlots = [] {
        const size_t fit = (227 * 1024 - kFixed) / SA_BYTES;
        return fit < (size_t)A_SLOTS_MAX ? (int)fit : A_SLOTS_MAX;
    }();
    static_assert(kASlots >= 4, "A ring");
    static constexpr size_t kNeed = kFixed + kASlots * SA_BYTES;
    // alone on its SM: a second CTA would wait in tcgen05.alloc for the 512
    // columns, so the request is padded past half of the SM's shared memory
    static constexpr size_t kSmem = kNeed > 116 * 1024 ? kNeed : 116 * 1024;
    static_assert(64 * ND <= (int)S_TMEM, "group accumulators fit in TMEM");
    static_assert(2 * kSmem > 228 * 1024, "one CTA per SM");
    static_assert(kSmem <= 227 * 1024, "shared memory");
};

template <int NDA, int NDB>
__global__ void __launch_bounds__(kSlicedThreads, 1)
k_tc_sliced(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int m, int n, int kpad,
            float alpha, const int *ea, const int *fb, dfloat *D, int64_t ldd) {
    using Cfg = SlicedCfg<NDA, NDB>;
    constexpr int ND = Cfg::ND;
    extern __shared__ unsigned char smraw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = base;
    constexpr int A_SLOTS = Cfg::kASlots;
    unsigned char *sB = base + A_SLOTS * SA_BYTES;
    dfloat *stage = reinterpret_cast<dfloat *>(sB + 2 * Cfg::kBStage);   // BM x kHalfLd
    SCtl *ctl = (SCtl *)(sB + 2 * Cfg::kBStage + STAGE_BYTES);
    volatile int *abort = &ctl->abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkt = kpad / BK;
    const int ntm = (m + BM - 1) / BM, ntn = (n + SBN - 1) / SBN;
    const int ntiles = ntm * ntn;
    // Tile order: the CTAs in flight walk the M tiles of a few N columns when
    // the M side is the narrow operand (a one- or two-digit multiplier), so the wide
    // operand's digit slices of those columns are shared through L2 and the
    // narrow one is what gets re-read; otherwise the N tiles of a few M rows.
    auto tile_m = [&](int tile) { return NDA < NDB ? tile % ntm : tile / ntn; };
    auto tile_n = [&](int tile) { return NDA < NDB ? tile / ntm : tile % ntn; };

    if (threadIdx.x == 0) {
        for (int s = 0; s < A_SLOTS; ++s) {
            mbar_init(&ctl->afull[s], 1);
            mbar_init(&ctl->aempty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&ctl->bfull[s], 1);
            mbar_init(&ctl->bempty[s], 1);
        }
        mbar_init(&ctl->tfull, 1);
        mbar_init(&ctl->tempty, 4);
        mbar_init(&ctl->drain, 1);
        ctl->abort = 0;
        ctl->issued_a = 0;
        ctl->issued_b = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(&ctl->tmem)),
                     "r"(S_TMEM)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = ctl->tmem;

    if (warp == 4) {
        // ---------------- producer ----------------
        if (lane == 0) {
            int ai = 0, bi = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                const int m0 = tile_m(tile) * BM, n0 = tile_n(tile) * SBN;
                for (int kt = 0; kt < nkt && ok; ++kt, ++bi) {
                    const int bs = bi & 1;
                    if (bi >= 2 && !mbar_wait(&ctl->bempty[bs], (uint32_t)((bi >> 1) & 1) ^ 1u, abort)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&ctl->bfull[bs], Cfg::kBStage);
                    for (int u = 0; u < NDB; ++u)
                        tma_2d(sB + bs * Cfg::kBStage + u * SBD_BYTES, &tmB, &ctl->bfull[bs], u * kpad + kt * BK, n0);
                    ctl->issued_b = bi + 1;
                    for (int t = 0; t < NDA; ++t, ++ai) {
                        const int slot = ai % A_SLOTS;
                        if (ai >= A_SLOTS &&
                            !mbar_wait(&ctl->aempty[slot], (uint32_t)((ai / A_SLOTS) & 1) ^ 1u, abort)) {
                            ok = false;
                            break;
                        }
                        mbar_expect_tx(&ctl->afull[slot], SA_BYTES);
                        tma_2d(sA + slot * SA_BYTES, &tmA, &ctl->afull[slot], t * kpad + kt * BK, m0);
                        ctl->issued_a = ai + 1;
                    }
                }
            }
            if (!ok) *abort = 1;
        }
        __syncwarp();
    } else if (warp == 5) {
        // ---------------- MMA issue ----------------
        if (lane == 0) {
            bool ok = true;
            int ai = 0, bi = 0, tc = 0;
            for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++tc) {
                // the previous tile's accumulators must have been read out
                if (tc > 0 && !mbar_wait(&ctl->tempty, (uint32_t)((tc - 1) & 1), abort)) {
                    ok = false;
                    break;
                }
                fence_after();
                for (int kt = 0; kt < nkt && ok; ++kt, ++bi) {
                    const int bs = bi & 1;
                    if (!mbar_wait(&ctl->bfull[bs], (uint32_t)((bi >> 1) & 1), abort)) {
                        ok = false;
                        break;
                    }
                    const uint32_t bbase = sa(sB + bs * Cfg::kBStage);
#pragma unroll
                    for (int t = 0; t < NDA; ++t) {
                        const int slot = ai % A_SLOTS;
                        if (!ok || !mbar_wait(&ctl->afull[slot], (uint32_t)((ai / A_SLOTS) & 1), abort)) {
                            ok = false;
                            continue;
                        }
                        ++ai;
                        fence_after();
                        const uint64_t ad = sdesc(sa(sA + slot * SA_BYTES));
                        const int nu = NDB < ND - t ? NDB : ND - t;   // B digits 0 .. nu - 1 (groups t .. t + nu - 1)
                        const int nrows = SBN * nu;
                        // the tile's first MMA into a group overwrites it: digit 0 opens
                        // groups 0 .. nu - 1; a later digit opens its last group when
                        // NDB <= ND - t (never when NDB = ND)
                        const int fresh = (t == 0) ? 0 : (NDB <= ND - t ? nrows - SBN : nrows);
#pragma unroll
                        for (int k = 0; k < BK / UMMA_K; ++k) {
                            const bool first = kt == 0 && k == 0;
#pragma unroll
                            for (int c0 = 0; c0 < nrows; c0 += 256) {
                                const int c1 = nrows - c0 < 256 ? c0 + (nrows - c0) : c0 + 256;
                                if (first && fresh > c0 && fresh < c1) {
                                    // split at the fresh group: accumulate below, overwrite from it on
                                    mma_n(tmem + (uint32_t)(SBN * t + c0), ad + (uint64_t)(k * 2),
                                          sdesc(bbase + (uint32_t)c0 * 128u) + (uint64_t)(k * 2), idesc_n(fresh - c0),
                                          1u);
                                    mma_n(tmem + (uint32_t)(SBN * t + fresh), ad + (uint64_t)(k * 2),
                                          sdesc(bbase + (uint32_t)fresh * 128u) + (uint64_t)(k * 2),
                                          idesc_n(c1 - fresh), 0u);
                                } else {
                                    const uint32_t acc = (first && c0 >= fresh) ? 0u : 1u;
                                    mma_n(tmem + (uint32_t)(SBN * t + c0), ad + (uint64_t)(k * 2),
                                          sdesc(bbase + (uint32_t)c0 * 128u) + (uint64_t)(k * 2), idesc_n(c1 - c0),
                                          acc);
                                }
                            }
                        }
                        commit(&ctl->aempty[slot]);
                    }
                    if (ok) commit(&ctl->bempty[bs]);
                }
                if (ok) commit(&ctl->tfull);
            }
            if (!ok) *abort = 1;
        }
        __syncwarp();
    } else {
        // ---------------- epilogue (warps 0-3, TMEM lanes 0-127) ----------------
        const int r = warp * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        int tc = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++tc) {
            const int m0 = tile_m(tile) * BM, n0 = tile_n(tile) * SBN;
            const int row = m0 + r;
            // this tile's rows of D into L2 while its MMAs run
            if (row < m && n0 < n) {
                const char *rp = reinterpret_cast<const char *>(D + (int64_t)row * ldd + n0);
                const int bytes = (n - n0 < SBN ? n - n0 : SBN) * (int)sizeof(dfloat);
                for (int b = 0; b < bytes; b += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(rp + b));
            }
            epi_sync();                        // every thread is done with the previous tile's cs
            if (r < SBN) {
                const int col = n0 + r;
                ctl->cs[r] = col < n ? ldexpf(alpha, fb[col]) : 0.0f;
            }
            const float rs = ldexpf(1.0f, (row < m ? ea[row] : 0) - 7 * ND);
            const bool ready = mbar_wait_sleep(&ctl->tfull, (uint32_t)(tc & 1), abort);
            if (!ready) *abort = 1;
            fence_after();
            // one decision for all four warps (they share a named barrier)
            epi_sync();
            if (r == 0) ctl->epi_go = *abort ? 0 : 1;
            epi_sync();
            if (!ctl->epi_go) break;
            // S as double-float, hi and lo parts of column pairs (2i, 2i + 1)
            float2 SH[2][16], SL[2][16];
            uint32_t q[32];
            const float2 w128 = make_float2(128.0f, 128.0f), w1 = make_float2(1.0f, 1.0f);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                // Horner over the groups, largest weight first: S = 2^7 S + P_g.  The
                // P_g are integers below 2^24 and the partial sums integers below
                // 2^60: exact as double-float up to 48 bits, all on the FP32 pipe,
                // two columns per instruction.
                tmem_ld32(lane_addr + (uint32_t)(32 * h), q);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    SH[h][i] = make_float2(__uint_as_float(q[2 * i]), __uint_as_float(q[2 * i + 1]));
                    SL[h][i] = make_float2(0.0f, 0.0f);
                }
#pragma unroll 1
                for (int g = 1; g < ND - 1; ++g) {
                    tmem_ld32(lane_addr + (uint32_t)(SBN * g + 32 * h), q);
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        horner2(SH[h][i], SL[h][i],
                                make_float2(__uint_as_float(q[2 * i]), __uint_as_float(q[2 * i + 1])), w128);
                }
                tmem_ld32(lane_addr + (uint32_t)(SBN * (ND - 1) + 32 * h), q);   // the last group: 2^-7
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    horner2(SH[h][i], SL[h][i],
                            make_float2(__uint_as_float(q[2 * i]) * 0.0078125f,
                                        __uint_as_float(q[2 * i + 1]) * 0.0078125f),
                            w1);
            }
            // TMEM is free for the next tile's MMAs
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl->tempty);
            // D += 2^{e_i - 7 ND} alpha 2^{f_j} S (two exact power-of-two scalings),
            // half a tile at a time through shared memory so the read-modify-write
            // of D runs along rows, eight rows' loads in flight per warp
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                epi_sync();                    // the staging area is free
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float c0 = ctl->cs[32 * h + 2 * i], c1 = ctl->cs[32 * h + 2 * i + 1];
                    dfloat a0, a1;
                    a0.hi = (SH[h][i].x * rs) * c0;
                    a0.lo = (SL[h][i].x * rs) * c0;
                    a1.hi = (SH[h][i].y * rs) * c1;
                    a1.lo = (SL[h][i].y * rs) * c1;
                    stage[r * kHalfLd + 2 * i] = a0;
                    stage[r * kHalfLd + 2 * i + 1] = a1;
                }
                epi_sync();
                const int col = n0 + 32 * h + lane;
                for (int r0 = warp * 32; r0 < warp * 32 + 32; r0 += 8) {
                    dfloat d[8];
#pragma unroll
                    for (int qq = 0; qq < 8; ++qq) {
                        const int rw = m0 + r0 + qq;
                        d[qq] = (rw < m && col < n) ? D[(int64_t)rw * ldd + col] : dfloat(0.0f);
                    }
#pragma unroll
                    for (int qq = 0; qq < 8; ++qq) {
                        const int rw = m0 + r0 + qq;
                        if (rw < m && col < n) D[(int64_t)rw * ldd + col] = d[qq] + stage[(r0 + qq) * kHalfLd + lane];
                    }
                }
            }
        }
    }

    fence_before();
    __syncthreads();
    if (ctl->abort) {
        // drain the copies still in flight before the CTA's shared memory goes away
        if (threadIdx.x == 128) {
            atomicExch(&g_tc_timeout, 1);
            int dummy = 0;
            const int ia = ctl->issued_a, ib = ctl->issued_b;
            for (int i = (ia > A_SLOTS ? ia - A_SLOTS : 0); i < ia; ++i)
                mbar_wait(&ctl->afull[i % A_SLOTS], (uint32_t)((i / A_SLOTS) & 1), (volatile int *)&dummy);
            for (int i = (ib > 2 ? ib - 2 : 0); i < ib; ++i)
                mbar_wait(&ctl->bfull[i & 1], (uint32_t)((i >> 1) & 1), (volatile int *)&dummy);
        }
        if (threadIdx.x == 160) {     // the MMA thread: wait for its MMAs still in flight
            int dummy = 0;
            commit(&ctl->drain);
            mbar_wait(&ctl->drain, 0, (volatile int *)&dummy);
        }
        __syncthreads();
    }
    if (warp == 5)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S_TMEM) : "memory");
}

// SMs the persistent sliced product leaves free (a concurrent one-CTA
// kernel of the factorization's look-ahead runs there); per host thread.
thread_local int tl_sliced_spare = 0;

// Optional CUDA-event timing of every k_tc_sliced launch (genp_profile_*).
struct TcProfile {
    bool on = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    std::vector<double> fl;       // flops of each recorded launch (as issued)
    std::vector<double> alg;      // its algorithmic flops (the product's own 2 m n K)
    size_t used = 0;
    double flops = 0.0;
};
TcProfile &tc_profile() {
    static TcProfile p;
    return p;
}
// Events around one launch of `flops` flops, or nullptr when profiling is off.
thread_local bool tl_profile_suspended = false;

std::pair<cudaEvent_t, cudaEvent_t> *profile_slot(double flops, double alg) {
    TcProfile &p = tc_profile();
    if (!p.on || tl_profile_suspended) return nullptr;
    if (p.used == p.ev.size()) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess) return nullptr;
        if (cudaEventCreate(&b) != cudaSuccess) {
            cudaEventDestroy(a);
            return nullptr;
        }
        p.ev.emplace_back(a, b);
        p.fl.push_back(0.0);
        p.alg.push_back(0.0);
    }
    p.fl[p.used] = flops;
    p.alg[p.used] = alg;
    p.flops += flops;
    return &p.ev[p.used++];
}

// The other kernel classes (genp::ProfClass), kept apart from the
// tensor-core list so that genp_profile_launches keeps its meaning.
struct ClassProfile {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    std::vector<double> work;
    std::vector<int> cls;
    size_t used = 0;
};
ClassProfile &class_profile() {
    static ClassProfile p;
    return p;
}

template <int NDA, int NDB>
cudaError_t launch_sliced(const CUtensorMap &ma, const CUtensorMap &mb, int64_t m, int64_t n, int64_t kpad,
                          float alpha, const int *ea, const int *fb, dfloat *D, int64_t ldd, cudaStream_t s) {
    using Cfg = SlicedCfg<NDA, NDB>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_tc_sliced<NDA, NDB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Cfg::kSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    // persistent: one CTA per SM, never more CTAs than tiles
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 148;
    }
    const int64_t tiles = cdiv(m, BM) * cdiv(n, SBN);
    if (tiles > INT32_MAX) return cudaErrorInvalidValue;
    const int use = sms - tl_sliced_spare > 0 ? sms - tl_sliced_spare : 1;
    const unsigned grid = (unsigned)(tiles < use ? tiles : use);
    auto *ev = profile_slot(2.0 * (double)m * (double)n * (double)kpad * Cfg::kPairs,
                            2.0 * (double)m * (double)n * (double)kpad);
    if (ev) cudaEventRecord(ev->first, s);
    note_launch();
    k_tc_sliced<NDA, NDB><<<grid, kSlicedThreads, Cfg::kSmem, s>>>(ma, mb, (int)m, (int)n, (int)kpad, alpha, ea, fb,
                                                                     D, ldd);
    if (ev) cudaEventRecord(ev->second, s);
    return cudaGetLastError();
}

}  // namespace

bool make_map_8b(CUtensorMap *map, const void *ptr, int64_t rows, int64_t cols, int64_t ld, int box_cols,
                 int box_rows) {
    auto fn = encoder();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 8)};
    cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void *>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sliced_spare_sms(int k) {
    const int prev = tl_sliced_spare;
    tl_sliced_spare = k;
    return prev;
}

cudaError_t tc_gemm_sliced(int nd, int64_t m, int64_t n, int64_t kpad, float alpha, const __nv_bfloat16 *Aq,
                           int64_t lda, const __nv_bfloat16 *Bq, int64_t ldb, const int *ea, const int *fb, dfloat *D,
                           int64_t ldd, cudaStream_t s) {
    return tc_gemm_sliced2(nd, nd, m, n, kpad, alpha, Aq, lda, Bq, ldb, ea, fb, D, ldd, s);
}

cudaError_t tc_gemm_sliced2(int nda, int ndb, int64_t m, int64_t n, int64_t kpad, float alpha,
                            const __nv_bfloat16 *Aq, int64_t lda, const __nv_bfloat16 *Bq, int64_t ldb, const int *ea,
                            const int *fb, dfloat *D, int64_t ldd, cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    const bool sym = nda == ndb && sliced::supported(nda);
    // a one- or two-digit M side (a multiplier on the sliced grid), the wide operand along N
    const bool narrow = (nda == 1 || nda == 2) && ndb >= 5 && ndb <= 7;
    if (!sym && !narrow) return cudaErrorInvalidValue;
    const int64_t kmax = nda <= 2 ? kSlicedChunk2 : kSlicedChunk;
    if (kpad <= 0 || kpad % BK || kpad > kmax || m > INT32_MAX || n > INT32_MAX) return cudaErrorInvalidValue;
    if ((lda % 8) || (ldb % 8) || ((uintptr_t)Aq % 16) || ((uintptr_t)Bq % 16)) return cudaErrorInvalidValue;
    const int64_t kqa = (int64_t)nda * kpad, kqb = (int64_t)ndb * kpad;
    if (lda < kqa || ldb < kqb) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!make_map(&ma, Aq, m, kqa, lda, BM) || !make_map(&mb, Bq, n, kqb, ldb, SBN)) return cudaErrorInvalidValue;
    switch (nda * 8 + ndb) {
        case 3 * 9: return launch_sliced<3, 3>(ma, mb, m, n, kpad, alpha, ea, fb, D, ldd, s);
        case 4 * 9: return launch_sliced<4, 4>(ma, mb, m, n, kpad, alpha, ea, fb, D, ldd, s);
        case 5 * 9: return launch_sliced<5, 5>(ma, mb, m, n, kpad, alpha, ea, fb, D, ldd, s);
        case 6 * 9: return launch_sliced<6, 6>(ma, mb, m, n, kpad, alpha, ea, fb, D, ldd, s);
        case 7 * 9: return launch_sliced<7, 7>(ma, mb, m, n, kpad, alpha, ea, fb, D, ldd, s);
        case 1 * 8 + 5: return launch_sliced<1, 5>(ma, mb, m, n, kpad, alpha, ea, fb, D, ldd, s);
        case 1 * 8 + 6: return launch_sliced<1, 6>(ma, mb, m, n, kpad, alpha, ea, fb, D, ldd, s);
        case 1 * 8 + 7: return launch_sliced<1, 7>(ma, mb, m, n, kpad, alpha, ea, fb, D, ldd, s);
        case 2 * 8 + 5: return launch_sliced<2, 5>(ma, mb, m, n, kpad, alpha, ea, fb, D, ldd, s);
        case 2 * 8 + 6: return launch_sliced<2, 6>(ma, mb, m, n, kpad, alpha, ea, fb, D, ldd, s);
        case 2 * 8 + 7: return launch_sliced<2, 7>(ma, mb, m, n, kpad, alpha, ea, fb, D, ldd, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t tc_gemm_bf16(int64_t m, int64_t n, int64_t K, float alpha, const __nv_bfloat16 *A, int64_t lda,
                         const __nv_bfloat16 *Bt, int64_t ldb, float beta, const float *Cin, int64_t ldci, float *D,
                         int64_t ldd, const int *skip, cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    if (K <= 0 || m > INT32_MAX || n > INT32_MAX || K > INT32_MAX) return cudaErrorInvalidValue;
    // TMA: 16-byte aligned bases and row strides
    if ((lda % 8) || (ldb % 8) || ((uintptr_t)A % 16) || ((uintptr_t)Bt % 16)) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, m, K, lda, BM) || !make_map(&mb, Bt, n, K, ldb, BN)) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e =
            cudaFuncSetAttribute(k_tc_gemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((unsigned)cdiv(n, BN), (unsigned)cdiv(m, BM));
    if (grid.y > 65535u) return cudaErrorInvalidValue;
    const int vec = ((uintptr_t)D % 16 == 0) && (ldd % 4 == 0) &&
                    (beta == 0.0f || ((uintptr_t)Cin % 16 == 0 && ldci % 4 == 0));
    note_launch();
    k_tc_gemm<false><<<grid, 128, kSmem, s>>>(ma, mb, (int)m, (int)n, (int)K, alpha, beta, Cin, ldci, D, ldd, vec,
                                              skip, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t tc_gemm_e4m3(int64_t m, int64_t n, int64_t K, float alpha, const uint8_t *A, int64_t lda, const float *sa,
                         const uint8_t *Bt, int64_t ldb, const float *sb, float beta, const float *Cin, int64_t ldci,
                         float *D, int64_t ldd, cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    if (K <= 0 || m > INT32_MAX || n > INT32_MAX || K > (int64_t)kQMaxKt * QBK) return cudaErrorInvalidValue;
    // TMA: 16-byte aligned bases and row strides
    if ((lda % 16) || (ldb % 16) || ((uintptr_t)A % 16) || ((uintptr_t)Bt % 16)) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!make_map_u8(&ma, A, m, K, lda) || !make_map_u8(&mb, Bt, n, K, ldb)) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_tc_e4m3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kQSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_tc_gemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((unsigned)cdiv(n, BN), (unsigned)cdiv(m, BM));
    if (grid.y > 65535u) return cudaErrorInvalidValue;
    const int vec = ((uintptr_t)D % 16 == 0) && (ldd % 4 == 0) &&
                    (beta == 0.0f || ((uintptr_t)Cin % 16 == 0 && ldci % 4 == 0));
    auto *ev = profile_slot(2.0 * (double)m * (double)n * (double)K, 2.0 * (double)m * (double)n * (double)K);
    if (ev) cudaEventRecord(ev->first, s);
    note_launch();
    if (K <= QBK)   // one k-tile: the scale product joins alpha, two CTAs per SM
        k_tc_gemm<true><<<grid, 128, kSmem, s>>>(ma, mb, (int)m, (int)n, (int)K, alpha, beta, Cin, ldci, D, ldd, vec,
                                                 nullptr, sa, sb);
    else
        k_tc_e4m3<<<grid, kQThreads, kQSmem, s>>>(ma, mb, (int)m, (int)n, (int)K, alpha, sa, sb, beta, Cin, ldci, D,
                                                  ldd, vec);
    if (ev) cudaEventRecord(ev->second, s);
    return cudaGetLastError();
}

void tc_profile_enable(bool on) {
    TcProfile &p = tc_profile();
    p.on = on;
    p.used = 0;
    p.flops = 0.0;
    class_profile().used = 0;
    trsv_skipped_count(true);
    gemv_skipped_count(true);
}

void profile_suspend(bool on) { tl_profile_suspended = on; }

std::pair<cudaEvent_t, cudaEvent_t> *profile_class_slot(int c, double work) {
    if (!tc_profile().on || tl_profile_suspended || c <= 0 || c >= kProfClasses) return nullptr;
    ClassProfile &p = class_profile();
    if (p.used == p.ev.size()) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess) return nullptr;
        if (cudaEventCreate(&b) != cudaSuccess) {
            cudaEventDestroy(a);
            return nullptr;
        }
        p.ev.emplace_back(a, b);
        p.work.push_back(0.0);
        p.cls.push_back(0);
    }
    p.work[p.used] = work;
    p.cls[p.used] = c;
    return &p.ev[p.used++];
}

int profile_class_read(int c, double *ms, double *work) {
    double t_sum = 0.0, w_sum = 0.0;
    int count = 0;
    if (c == kProfTensor) {   // the tensor-core list, counted by algorithmic flops
        TcProfile &q = tc_profile();
        for (size_t i = 0; i < q.used; ++i) {
            if (cudaEventSynchronize(q.ev[i].second) != cudaSuccess) return -1;
            float t = 0.0f;
            if (cudaEventElapsedTime(&t, q.ev[i].first, q.ev[i].second) != cudaSuccess) return -1;
            t_sum += t;
            w_sum += q.alg[i];
            ++count;
        }
        *ms = t_sum;
        *work = w_sum;
        return count;
    }
    ClassProfile &p = class_profile();
    for (size_t i = 0; i < p.used; ++i) {
        if (p.cls[i] != c) continue;
        if (cudaEventSynchronize(p.ev[i].second) != cudaSuccess) return -1;
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, p.ev[i].first, p.ev[i].second) != cudaSuccess) return -1;
        t_sum += t;
        w_sum += p.work[i];
        ++count;
    }
    // launches that returned on their skip flag did no work; within a class
    // of one workload the launches carry equal work, so scale by the share
    // that ran
    const unsigned int skipped = c == kProfTrsv ? trsv_skipped_count(false)
                                                : (c == kProfGemv ? gemv_skipped_count(false) : 0u);
    if (count > 0) w_sum *= (double)(count - (int)(skipped < (unsigned)count ? skipped : count)) / count;
    *ms = t_sum;
    *work = w_sum;
    return count;
}

int tc_profile_launches(double *ms, double *flops, int cap) {
    TcProfile &p = tc_profile();
    const int count = (int)p.used;
    for (int i = 0; i < count && i < cap; ++i) {
        if (cudaEventSynchronize(p.ev[i].second) != cudaSuccess) return -1;
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, p.ev[i].first, p.ev[i].second) != cudaSuccess) return -1;
        if (ms) ms[i] = t;
        if (flops) flops[i] = p.fl[i];
    }
    return count;
}

int tc_profile_read(double *ms, double *flops) {
    TcProfile &p = tc_profile();
    double total = 0.0;
    for (size_t i = 0; i < p.used; ++i) {
        if (cudaEventSynchronize(p.ev[i].second) != cudaSuccess) return -1;
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, p.ev[i].first, p.ev[i].second) != cudaSuccess) return -1;
        total += t;
    }
    *ms = total;
    *flops = p.flops;
    const int count = (int)p.used;
    p.used = 0;
    p.flops = 0.0;
    return count;
}

int tc_timeout_flag(bool reset) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_timeout, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    if (reset && v) {
        int z = 0;
        cudaMemcpyToSymbol(g_tc_timeout, &z, sizeof(int));
    }
    return v;
}

}  // namespace genp
