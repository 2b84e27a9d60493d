// batched_r8.cu -- the batched kernels for up to 8 right-hand sides.
#include "batched_impl.cuh"

GENP_BATCHED_INSTANCE(8)
