// Kernels for groups of 8 threads x 4 words per thread (32 words, 1024 bits), 256 threads per block.
#include "mp_kernels.cuh"
MPG_DEFINE_SHAPE(8, 4, 256)
