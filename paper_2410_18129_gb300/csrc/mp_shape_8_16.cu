// Kernels for groups of 8 threads x 16 words per thread (128 words, 4096 bits), 128 threads per block.
#include "mp_kara.cuh"
MPG_DEFINE_SHAPE_KARA(8, 16, 128, 8, 128)
// Karatsuba: three half products on groups of 8 threads x 8 words, 128 threads per block.
