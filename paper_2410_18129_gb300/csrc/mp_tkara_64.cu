// 2048-bit class (64 words) in the Karatsuba form: half shape 4 threads x 8 words
#include "mp_tkara.cuh"
MPG_DEFINE_TKARA(64, 4, 8, 64)
