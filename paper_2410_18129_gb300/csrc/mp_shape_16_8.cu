// Kernels for groups of 16 threads x 8 words per thread (128 words, 4096 bits), 256 threads per
// block; the truncated and classical Montgomery kernels role-swapped in 512-thread blocks of 32
// instances.
#include "mp_kernels.cuh"
#include "mp_swap.cuh"
#ifdef MPG_LANE_ONLY
MPG_DEFINE_SHAPE(16, 8, 256)
#else
MPG_DEFINE_SHAPE_SWAP(16, 8, 256)
#endif
