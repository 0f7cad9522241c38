// Kernels for groups of 8 threads x 12 words per thread (96 words, 3072 bits), 128 threads per
// block; the truncated and classical Montgomery kernels and the products role-swapped in
// 256-thread blocks of 32 instances (two per SM: 128 registers per thread for the 12-word blocks'
// accumulators; Karatsuba: three half products of 8 roles x 6 words).
#include "mp_swap_prod.cuh"
#ifdef MPG_LANE_ONLY
MPG_DEFINE_SHAPE_KARA(8, 12, 128, 6, 128)
#else
MPG_DEFINE_SHAPE_SWAP_ALL(8, 12, 128, 8, 12, 8, 6)
#endif
