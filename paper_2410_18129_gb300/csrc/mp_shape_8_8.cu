// Kernels for groups of 8 threads x 8 words per thread (64 words, 2048 bits), 256 threads per block.
#include "mp_kernels.cuh"
MPG_DEFINE_SHAPE(8, 8, 256)
