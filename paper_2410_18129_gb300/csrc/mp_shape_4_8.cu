// Kernels for groups of 4 threads x 8 words per thread (32 words, 1024 bits), 256 threads per block;
// the truncated and classical Montgomery kernels role-swapped in 128-thread blocks of 32 instances.
#include "mp_kara.cuh"
#include "mp_swap.cuh"
#ifdef MPG_LANE_ONLY
MPG_DEFINE_SHAPE_KARA(4, 8, 256, 4, 256)
#else
MPG_DEFINE_SHAPE_KARA_SWAP(4, 8, 256, 4, 256)
#endif
// Karatsuba: three half products on groups of 4 threads x 4 words.
