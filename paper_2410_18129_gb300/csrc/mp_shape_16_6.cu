// Kernels for groups of 16 threads x 6 words per thread (96 words, 3072 bits), 256 threads per block.
#include "mp_kernels.cuh"
MPG_DEFINE_SHAPE(16, 6, 256)
