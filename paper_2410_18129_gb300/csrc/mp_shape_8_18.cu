// Kernels for groups of 8 threads x 18 words per thread (144 words, 4608 bits), 128 threads per block.
#include "mp_kara.cuh"
MPG_DEFINE_SHAPE_KARA(8, 18, 128, 9, 128)
// Karatsuba: three half products on groups of 8 threads x 9 words, 128 threads per block.
