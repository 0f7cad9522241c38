// Kernels for groups of 8 threads x 12 words per thread (96 words, 3072 bits), 128 threads per block.
#include "mp_kernels.cuh"
MPG_DEFINE_SHAPE(8, 12, 128)
