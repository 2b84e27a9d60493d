// batched_r16.cu -- the batched kernels for up to 16 right-hand sides.
#include "batched_impl.cuh"

GENP_BATCHED_INSTANCE(16)
