// batched_r2.cu -- the batched kernels for up to 2 right-hand sides.
#include "batched_impl.cuh"

GENP_BATCHED_INSTANCE(2)
