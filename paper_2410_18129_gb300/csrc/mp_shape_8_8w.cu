// Kernels for 8 threads x 8 words (64 words, 2048 bits) with thread t of every instance in
// warp t of a block of 8 warps (lane = instance, 32 instances per block).
#include "mp_kernels.cuh"
MPG_DEFINE_SHAPE_W(8, 8)
