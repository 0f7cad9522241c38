// Kernels for groups of 4 threads x 8 words per thread (32 words, 1024 bits), 256 threads per block;
// the truncated and classical Montgomery kernels and the products role-swapped in 128-thread
// blocks of 32 instances (Karatsuba: three half products of 4 roles x 4 words).
#include "mp_swap_prod.cuh"
#ifdef MPG_LANE_ONLY
MPG_DEFINE_SHAPE_KARA(4, 8, 256, 4, 256)
#else
MPG_DEFINE_SHAPE_SWAP_ALL(4, 8, 256, 4, 8, 4, 4)
#endif
