// Library-internal declarations shared by the translation units of libmpgpu
// (not part of the C ABI).
#pragma once
#include <cstddef>
#include <cstdint>
#include "mp_kernels.cuh"
#include "../../include/mpgpu.h"

struct mont_ctx {
    size_t batch;
    uint32_t bits, n, np;
    mp_layout layout;
    cudaStream_t stream;                           // stream of mont_ctx_init: allocation and free
    uint32_t *mem;                                 // one allocation for everything below
    uint32_t *N, *NI, *R1, *R2, *K;                // internal: interleaved, np words
    uint32_t *NI_api, *R1_api, *R2_api, *N_api;    // API layout, n words
    size_t api_words;                              // words of one API array
};

namespace mpg {
// fills the context fields of a kernel argument block
void ctx_args(KArgs &A, const mont_ctx *c);
// window used when the caller passes window = 0
uint32_t default_window(uint32_t bits);
// kernels of the size class of np words for reduction red (the selected shape; a lane-mapped one
// for the word-serial reduction), or null
const ShapeOps *shape_for_red_np(uint32_t np, int red);
}  // namespace mpg
