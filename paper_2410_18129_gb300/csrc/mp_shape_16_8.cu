// Kernels for groups of 16 threads x 8 words per thread (128 words, 4096 bits), 256 threads per block.
#include "mp_kernels.cuh"
MPG_DEFINE_SHAPE(16, 8, 256)
