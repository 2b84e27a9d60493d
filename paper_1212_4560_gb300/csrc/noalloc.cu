// noalloc.cu -- an allocation-free way to draw the sparse +-1 multiplier.
//
// genp_make_multiplier allocates the multiplier's storage and the scratch
// for the Fisher-Yates swap draws with cudaMalloc.  Some callers cannot do
// that: code whose device memory is owned by another allocator (a framework
// pool that has already reserved the device's memory, or an application that
// maps all of its memory once at start-up) and code in a latency-critical
// loop that must not pay the device-wide synchronization cudaMalloc and
// cudaFree can cause.  genp_make_sparse_noalloc writes the same multiplier
// into buffers the caller already owns and keeps its scratch in the
// file-scope device array below, so the call allocates nothing.
//
// The array is a fixed GENP_NOALLOC_MAX_ENTRIES int32 (4 MiB) that every GPU
// which loads this library holds until the process exits.  Host code only
// sees a host-side stand-in for it, so its device address is looked up once
// per device with cudaGetSymbolAddress and that address is what the kernels
// get.
#include "genp_internal.cuh"

#include <mutex>

static __device__ __align__(256) int32_t g_noalloc_draws[GENP_NOALLOC_MAX_ENTRIES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int32_t *g_draws_ptr[kMaxDevices] = {};

// Device address of g_noalloc_draws on the current device (looked up on the
// first call per device, with that device current).
cudaError_t scratch_on_current_device(int32_t **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_draws_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_draws);
        if (e != cudaSuccess) return e;
        g_draws_ptr[dev] = static_cast<int32_t *>(p);
    }
    *out = g_draws_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" genp_status genp_make_sparse_noalloc(int64_t n, int nnz_per_col, uint64_t seed, uint64_t stream_id,
                                                int32_t *rows, int8_t *signs, int32_t *inv_rows, int8_t *inv_signs,
                                                void *cuda_stream) {
    if (n < 1 || nnz_per_col < 1 || nnz_per_col > 16) return GENP_ERR_ARG;
    if (!rows || !signs || !inv_rows || !inv_signs) return GENP_ERR_ARG;
    if (n * (int64_t)nnz_per_col > (int64_t)GENP_NOALLOC_MAX_ENTRIES) return GENP_ERR_ARG;  // beyond the scratch
    int32_t *draws = nullptr;
    if (scratch_on_current_device(&draws) != cudaSuccess) {
        cudaGetLastError();
        return GENP_ERR_CUDA;
    }
    // Every scratch entry the shuffle reads is written by the draw kernel of
    // this same call first, so nothing has to be cleared between calls.
    if (genp::launch_make_sparse(rows, signs, inv_rows, inv_signs, draws, n, nnz_per_col, seed, stream_id,
                                 static_cast<cudaStream_t>(cuda_stream)) != cudaSuccess) {
        cudaGetLastError();
        return GENP_ERR_CUDA;
    }
    return GENP_OK;
}
