// Kernels for groups of 8 threads x 8 words per thread (64 words, 2048 bits): products and the
// word-serial reduction lane-mapped in 288-thread blocks, the truncated and classical Montgomery
// kernels role-swapped in 256-thread blocks of 32 instances.
#include "mp_kara.cuh"
#include "mp_swap.cuh"
MPG_DEFINE_SHAPE_KARA_SWAP(8, 8, 288, 4, 256)
// Karatsuba: three half products on groups of 8 threads x 4 words, 256 threads per block.
