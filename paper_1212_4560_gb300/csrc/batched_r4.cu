// batched_r4.cu -- the batched kernels for up to 4 right-hand sides.
#include "batched_impl.cuh"

GENP_BATCHED_INSTANCE(4)
