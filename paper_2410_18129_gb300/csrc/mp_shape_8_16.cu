// Kernels for groups of 8 threads x 16 words per thread (128 words, 4096 bits), 128 threads per block.
#include "mp_kernels.cuh"
MPG_DEFINE_SHAPE(8, 16, 128)
