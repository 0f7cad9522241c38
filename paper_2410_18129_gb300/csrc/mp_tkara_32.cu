// 1024-bit class (32 words) in the Karatsuba form: half shape 2 threads x 8 words
#include "mp_tkara.cuh"
MPG_DEFINE_TKARA(32, 2, 8, 64)
