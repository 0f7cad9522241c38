// 3072-bit class (96 words) in the Karatsuba form: half shape 4 threads x 12 words
#include "mp_tkara.cuh"
MPG_DEFINE_TKARA(96, 4, 12, 64)
