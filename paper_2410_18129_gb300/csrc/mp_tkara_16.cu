// 512-bit class (16 words) in the Karatsuba form: half shape 2 threads x 4 words
#include "mp_tkara.cuh"
MPG_DEFINE_TKARA(16, 2, 4, 64)
