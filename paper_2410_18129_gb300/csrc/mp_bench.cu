// Integer-multiply microbenchmark: sets the roofline denominator (IMAD issue
// rate per SM per clock) from measurement instead of an assumed figure.
#include <cuda_runtime.h>
#include <cstdint>
#include <vector>
#include <algorithm>
#include "mp_limb.cuh"
#include "../../include/mpgpu.h"

using namespace mpg;

// mode 0: independent 32-bit multiply-adds (mad.lo.u32), 8 chains per thread
// mode 1: independent high-half multiply-adds (mad.hi.u32)
// mode 2: the library's 8x8 block product (mad.lo.cc / madc.hi.cc carry chains), 128 IMAD per call
// mode 3: 32-bit add-with-carry chains (add.cc / addc.cc), 8 words
__global__ void k_bench(int mode, int iters, uint32_t seed, uint32_t *sink, long long *cycles) {
    uint32_t a[8], b[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) { a[i] = seed * (threadIdx.x + 3 * i + 1); b[i] = seed ^ (i * 0x9e3779b9u + threadIdx.x); }
    __syncthreads();
    long long t0 = clock64();
    if (mode == 0) {
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int r = 0; r < 16; ++r) {
#pragma unroll
                for (int i = 0; i < 8; ++i) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[i]) : "r"(b[i]), "r"(b[(i + 1) & 7]));
            }
        }
    } else if (mode == 1) {
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int r = 0; r < 16; ++r) {
#pragma unroll
                for (int i = 0; i < 8; ++i) asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(a[i]) : "r"(b[i]), "r"(b[(i + 1) & 7]));
            }
        }
    } else if (mode == 2) {
        uint32_t P[16];
        for (int it = 0; it < iters; ++it) {
            block_mul<8>(P, a, b);
#pragma unroll
            for (int i = 0; i < 8; ++i) { a[i] ^= P[i]; b[i] += P[8 + i]; }
        }
    } else {
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                add_cc(a[0], b[0]);
#pragma unroll
                for (int i = 1; i < 8; ++i) addc_cc(a[i], b[i]);
            }
        }
    }
    __syncthreads();
    long long t1 = clock64();
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc ^= a[i] + b[i];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

extern "C" int mp_bench_imad(int mode, int iters, double *per_clk_per_sm, double *sm_mhz, void *stream) {
    if (mode < 0 || mode > 3 || iters <= 0 || !per_clk_per_sm) return MP_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MP_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MP_ERR_CUDA;
    const int threads = 1024;
    uint32_t *sink = nullptr;
    long long *cyc = nullptr;
    if (cudaMalloc(&sink, (size_t)sms * threads * 4) != cudaSuccess) return MP_ERR_NOMEM;
    if (cudaMalloc(&cyc, (size_t)sms * 8) != cudaSuccess) { cudaFree(sink); return MP_ERR_NOMEM; }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_bench<<<sms, threads, 0, st>>>(mode, 1, 12345u, sink, cyc);   // warm-up
    cudaEventRecord(e0, st);
    k_bench<<<sms, threads, 0, st>>>(mode, iters, 12345u, sink, cyc);
    cudaEventRecord(e1, st);
    int rc = (cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess) ? MP_OK : MP_ERR_CUDA;
    if (rc == MP_OK) {
        std::vector<long long> c(sms);
        cudaMemcpy(c.data(), cyc, (size_t)sms * 8, cudaMemcpyDeviceToHost);
        std::sort(c.begin(), c.end());
        const double med = (double)c[sms / 2];
        const double per_thread = mode == 2 ? 128.0 * iters : mode == 3 ? 128.0 * iters : 128.0 * iters;
        *per_clk_per_sm = per_thread * threads / med;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (sm_mhz) *sm_mhz = (double)c[sms - 1] / (ms * 1e3);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    cudaFree(cyc);
    return rc;
}
