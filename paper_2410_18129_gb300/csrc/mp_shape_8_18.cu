// Kernels for groups of 8 threads x 18 words per thread (144 words, 4608 bits), 128 threads per block.
#include "mp_kernels.cuh"
MPG_DEFINE_SHAPE(8, 18, 128)
