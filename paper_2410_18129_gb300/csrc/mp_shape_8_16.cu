// Kernels for groups of 8 threads x 16 words per thread (128 words, 4096 bits), 128 threads per
// block; the truncated and classical Montgomery kernels and the products role-swapped in
// 256-thread blocks of 32 instances (Karatsuba: three half products of 8 roles x 8 words).
#include "mp_swap_prod.cuh"
#ifdef MPG_LANE_ONLY
MPG_DEFINE_SHAPE_KARA(8, 16, 128, 8, 128)
#else
MPG_DEFINE_SHAPE_SWAP_ALL(8, 16, 128, 8, 16, 8, 8)
#endif
