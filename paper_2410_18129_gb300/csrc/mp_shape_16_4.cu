// Kernels for groups of 16 threads x 4 words per thread (64 words, 2048 bits), 256 threads per block.
#include "mp_kernels.cuh"
MPG_DEFINE_SHAPE(16, 4, 256)
