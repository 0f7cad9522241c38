// Kernels for groups of 8 threads x 8 words per thread (64 words, 2048 bits), 256 threads per block.
#include "mp_kara.cuh"
MPG_DEFINE_SHAPE_KARA(8, 8, 288, 4, 256)
// Karatsuba: three half products on groups of 8 threads x 4 words, 256 threads per block.
