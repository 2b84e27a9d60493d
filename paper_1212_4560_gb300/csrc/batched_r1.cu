// batched_r1.cu -- the batched kernels for up to 1 right-hand sides.
#include "batched_impl.cuh"

GENP_BATCHED_INSTANCE(1)
