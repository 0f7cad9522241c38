// Kernels for groups of 8 threads x 12 words per thread (96 words, 3072 bits), 128 threads per block.
#include "mp_kara.cuh"
MPG_DEFINE_SHAPE_KARA(8, 12, 128, 6, 128)
// Karatsuba: three half products on groups of 8 threads x 6 words, 128 threads per block.
