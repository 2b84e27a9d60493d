// batched.cu -- dispatch of the batched kernels by right-hand-side class
// (the kernels themselves are in batched_impl.cuh, one translation unit per
// class).
#include "genp_internal.cuh"

namespace genp {
namespace {

int rhs_class(int nr) { return nr <= 1 ? 1 : nr <= 2 ? 2 : nr <= 4 ? 4 : nr <= 8 ? 8 : 16; }

}  // namespace

int batched_blocks_per_sm(int nr, int nmax) {
    switch (rhs_class(nr)) {
        case 1: return batched_blocks_per_sm_r1(nmax);
        case 2: return batched_blocks_per_sm_r2(nmax);
        case 4: return batched_blocks_per_sm_r4(nmax);
        case 8: return batched_blocks_per_sm_r8(nmax);
        default: return batched_blocks_per_sm_r16(nmax);
    }
}

// The Krylov copy of C, L^{-1} and U^{-1} (np^2 each), the basis
// ((K + 1) np NR), then the FP64 residual, last accepted x and its residual
// (np NR doubles each), np = nmax rounded up to 4 (16-byte offsets).
int64_t batched_scratch_stride(int nr, int nmax) {
    const int64_t NR = rhs_class(nr), np = (nmax + 3) & ~3;
    return 3 * np * np + (int64_t)(kBatchedKrylov + 1) * np * NR + 3 * 2 * np * NR;
}

cudaError_t launch_batched(BatchedArgs a, int grid, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    a.stride = batched_scratch_stride(a.nr, a.nmax);
    note_launch();
    switch (rhs_class(a.nr)) {
        case 1: return batched_launch_r1(a, grid, s);
        case 2: return batched_launch_r2(a, grid, s);
        case 4: return batched_launch_r4(a, grid, s);
        case 8: return batched_launch_r8(a, grid, s);
        default: return batched_launch_r16(a, grid, s);
    }
}

cudaError_t launch_batched_adjoint(BatchedArgs a, int grid, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    a.stride = batched_scratch_stride(a.nr, a.nmax);
    note_launch();
    switch (rhs_class(a.nr)) {
        case 1: return batched_adjoint_r1(a, grid, s);
        case 2: return batched_adjoint_r2(a, grid, s);
        case 4: return batched_adjoint_r4(a, grid, s);
        case 8: return batched_adjoint_r8(a, grid, s);
        default: return batched_adjoint_r16(a, grid, s);
    }
}

}  // namespace genp
