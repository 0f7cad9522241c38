// Kernels for groups of 2 threads x 4 words per thread (8 words, 256 bits), 256 threads per block.
#include "mp_kernels.cuh"
MPG_DEFINE_SHAPE(2, 4, 256)
