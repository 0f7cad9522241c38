// 4096-bit class (128 words) in the Karatsuba form: half shape 8 threads x 8 words
#include "mp_tkara.cuh"
MPG_DEFINE_TKARA(128, 8, 8, 64)
