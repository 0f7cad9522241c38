// Kernels for groups of 4 threads x 4 words per thread (16 words, 512 bits), 256 threads per block.
#include "mp_kernels.cuh"
MPG_DEFINE_SHAPE(4, 4, 256)
