// Kernels for groups of 8 threads x 8 words per thread (64 words, 2048 bits): the word-serial
// reduction lane-mapped in 288-thread blocks; the truncated and classical Montgomery kernels and
// the products role-swapped in 256-thread blocks of 32 instances (Karatsuba: three half products
// of 8 roles x 4 words).
#include "mp_swap_prod.cuh"
#ifdef MPG_LANE_ONLY
MPG_DEFINE_SHAPE_KARA(8, 8, 288, 4, 256)
#else
MPG_DEFINE_SHAPE_SWAP_ALL(8, 8, 288, 8, 8, 8, 4)
#endif
