// gemm_tc.cu -- BF16 tensor-core GEMM on sm_103a (tcgen05 + TMA + TMEM):
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
#include <cudaTypedefs.h>

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

__global__ void __launch_bounds__(128, 2)
k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int m, int n, int K,
          float alpha, float beta, const float *Cin, int64_t ldci, float *D, int64_t ldd, int vec, const int *skip) {
    if (skip && *skip) return;
    extern __shared__ unsigned char smraw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = base;
    unsigned char *sB = base + STAGES * A_BYTES;
    Ctl *ctl = (Ctl *)(sB + STAGES * B_BYTES);
    volatile int *abort = &ctl->abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int nk = (K + BK - 1) / BK;

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
            tma_2d(sA + s * A_BYTES, &tmA, &ctl->full[s], kt * BK, m0);
            tma_2d(sB + s * B_BYTES, &tmB, &ctl->full[s], kt * BK, n0);
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
            for (int k = 0; k < BK / UMMA_K; ++k)  // +32 bytes along K inside the swizzle atom
                mma(tmem, ad + (uint64_t)(k * 2), bd + (uint64_t)(k * 2), (kt > 0 || k > 0) ? 1u : 0u);
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

}  // namespace

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
        cudaError_t e = cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((unsigned)cdiv(n, BN), (unsigned)cdiv(m, BM));
    if (grid.y > 65535u) return cudaErrorInvalidValue;
    const int vec = ((uintptr_t)D % 16 == 0) && (ldd % 4 == 0) &&
                    (beta == 0.0f || ((uintptr_t)Cin % 16 == 0 && ldci % 4 == 0));
    note_launch();
    k_tc_gemm<<<grid, 128, kSmem, s>>>(ma, mb, (int)m, (int)n, (int)K, alpha, beta, Cin, ldci, D, ldd, vec, skip);
    return cudaGetLastError();
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
