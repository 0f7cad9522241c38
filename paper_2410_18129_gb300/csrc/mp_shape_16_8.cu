// Kernels for groups of 16 threads x 8 words per thread (128 words, 4096 bits), 256 threads per
// block; the truncated and classical Montgomery kernels role-swapped in 512-thread blocks of 32
// instances. Products run role-swapped on 8 roles x 16 words (measured 470 against 345 M mul/s
// on 16 x 8: the 16-word blocks carry less overhead per partial product), Karatsuba on half
// products of 8 roles x 8 words (464 M/s; 16 x 4: 408, 4 x 16: 309 with 8 warps per SM).
#include "mp_swap_prod.cuh"
#ifdef MPG_LANE_ONLY
MPG_DEFINE_SHAPE(16, 8, 256)
#else
MPG_DEFINE_SHAPE_SWAP_ALL(16, 8, 256, 8, 16, 8, 8)
#endif
