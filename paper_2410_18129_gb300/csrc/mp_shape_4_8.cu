// Kernels for groups of 4 threads x 8 words per thread (32 words, 1024 bits), 256 threads per block.
#include "mp_kernels.cuh"
MPG_DEFINE_SHAPE(4, 8, 256)
