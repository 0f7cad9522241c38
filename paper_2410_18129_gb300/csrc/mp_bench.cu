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
// mode 4: mad.wide.u32 (32x32+64 -> 64) chains fed by their own low word, counted as two multiply-adds
// mode 5: 8x8 block product from mad.wide.u32 plus 64-bit carry adds
// mode 6: two independent 8x8 carry-chain block products per iteration
// mode 7: mode 2 with 256 active threads per SM
// mode 8: 10x10 block of 26-bit digits summed into 64-bit columns with mad.wide.u32 (counted as 2 per product)
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
    } else if (mode == 3) {
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                add_cc(a[0], b[0]);
#pragma unroll
                for (int i = 1; i < 8; ++i) addc_cc(a[i], b[i]);
            }
        }
    } else if (mode == 4) {
        // 32x32+64 -> 64 multiply-adds (mad.wide.u32), 8 chains; counted as 2 (lo + hi). The
        // multiplier is the chain's previous low word, so no product can be precomputed.
        uint64_t w[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) w[i] = ((uint64_t)a[i] << 32) | b[i];
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int r = 0; r < 8; ++r) {
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(w[i]) : "r"((uint32_t)w[i]), "r"(a[(i + 1) & 7]));
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] ^= (uint32_t)w[i] ^ (uint32_t)(w[i] >> 32);
    } else if (mode == 5) {
        // 8x8 block product by operand scanning with mad.wide.u32: t = a_i*b_j + r + carry
        uint32_t P[16];
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int j = 0; j < 16; ++j) P[j] = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                uint32_t carry = 0;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    uint64_t t;
                    asm volatile("mad.wide.u32 %0, %1, %2, %3;" : "=l"(t) : "r"(a[i]), "r"(b[j]), "l"((uint64_t)P[i + j]));
                    t += carry;
                    P[i + j] = (uint32_t)t;
                    carry = (uint32_t)(t >> 32);
                }
                P[i + 8] = carry;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) { a[i] ^= P[i]; b[i] += P[8 + i]; }
        }
    } else if (mode == 6) {
        // two independent 8x8 carry-chain block products per iteration (instruction-level parallelism)
        uint32_t P[16], Q[16], c[8], d[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) { c[i] = a[i] * 3u + 1u; d[i] = b[i] ^ 0x55555555u; }
        for (int it = 0; it < iters; ++it) {
            block_mul<8>(P, a, b);
            block_mul<8>(Q, c, d);
#pragma unroll
            for (int i = 0; i < 8; ++i) { a[i] ^= P[i]; b[i] += P[8 + i]; c[i] ^= Q[i]; d[i] += Q[8 + i]; }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] ^= c[i] + d[i];
    } else {
        // mode 7: the 8x8 block product with 256 threads per SM (low occupancy)
        uint32_t P[16];
        if (threadIdx.x < 256) {
            for (int it = 0; it < iters; ++it) {
                block_mul<8>(P, a, b);
#pragma unroll
                for (int i = 0; i < 8; ++i) { a[i] ^= P[i]; b[i] += P[8 + i]; }
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


// mode 8 (own kernel: its 38 accumulator registers do not fit 1024 threads per SM)
__global__ void __launch_bounds__(512) k_bench_wide(int iters, uint32_t seed, uint32_t *sink, long long *cycles) {
    uint32_t x[10], y[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) { x[i] = (seed * (threadIdx.x + 3 * i + 1)) & 0x3ffffffu; y[i] = (seed ^ (i * 0x9e3779b9u + threadIdx.x)) & 0x3ffffffu; }
    uint64_t col[19];
#pragma unroll
    for (int c = 0; c < 19; ++c) col[c] = 0;
    __syncthreads();
    long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 10; ++i)
#pragma unroll
            for (int j = 0; j < 10; ++j)
                asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(col[i + j]) : "r"(x[i]), "r"(y[j]));
#pragma unroll
        for (int i = 0; i < 10; ++i) x[i] ^= (uint32_t)col[i] & 0x3ffffffu;
    }
    __syncthreads();
    long long t1 = clock64();
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < 19; ++c) acc ^= (uint32_t)col[c] ^ (uint32_t)(col[c] >> 32);
    sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// modes 9-12: block products summed into one running slot sum, as the Montgomery phases do
// (768 threads per SM, 24 warps):
//   9: 8x8 blocks, split-column accumulator (Acc3<8>)      10: 4x4 blocks, Acc3<4>
//  11: 8x8 blocks, block_mul + acc_add into one array      12: 4x4 blocks, block_mul + acc_add
// 128 multiply-adds (64 partial products) per iteration in every mode.
template <int MODE>
__global__ void __launch_bounds__(768, 1) k_bench_acc(int iters, uint32_t seed, uint32_t *sink, long long *cycles) {
    constexpr int B = (MODE == 9 || MODE == 11) ? 8 : 4;
    constexpr int REP = 64 / (B * B);
    uint32_t x[B], y[B];
#pragma unroll
    for (int i = 0; i < B; ++i) { x[i] = seed * (threadIdx.x + 3 * i + 1); y[i] = seed ^ (i * 0x9e3779b9u + threadIdx.x); }
    uint32_t fold = 0u;
    __syncthreads();
    long long t0 = clock64();
    if constexpr (MODE == 9 || MODE == 10) {
        Acc3<B> a;
        acc3_zero<B>(a);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int r = 0; r < REP; ++r) acc3_mac<B>(a, x, y);
#pragma unroll
            for (int i = 0; i < B; ++i) x[i] ^= a.E[i];
        }
        uint32_t V[2 * B + 2];
        acc3_value<B>(V, a);
#pragma unroll
        for (int j = 0; j < 2 * B + 2; ++j) fold ^= V[j];
    } else {
        uint32_t V[2 * B + 2];
#pragma unroll
        for (int j = 0; j < 2 * B + 2; ++j) V[j] = 0u;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int r = 0; r < REP; ++r) {
                uint32_t P[2 * B];
                block_mul<B>(P, x, y);
                acc_add<B>(V, P);
            }
#pragma unroll
            for (int i = 0; i < B; ++i) x[i] ^= V[i];
        }
#pragma unroll
        for (int j = 0; j < 2 * B + 2; ++j) fold ^= V[j];
    }
    __syncthreads();
    long long t1 = clock64();
#pragma unroll
    for (int i = 0; i < B; ++i) fold ^= x[i] + y[i];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = fold;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// modes 13-14: 4x4 blocks with 256 threads per SM (latency exposed): 13 one split accumulator,
// 14 two split accumulators taking alternate blocks (independent carry chains)
template <int MODE>
__global__ void __launch_bounds__(256, 1) k_bench_ilp(int iters, uint32_t seed, uint32_t *sink, long long *cycles) {
    constexpr int B = 4;
    uint32_t x[B], y[B];
#pragma unroll
    for (int i = 0; i < B; ++i) { x[i] = seed * (threadIdx.x + 3 * i + 1); y[i] = seed ^ (i * 0x9e3779b9u + threadIdx.x); }
    uint32_t fold = 0u;
    __syncthreads();
    long long t0 = clock64();
    Acc3<B> a, b;
    acc3_zero<B>(a);
    acc3_zero<B>(b);
    for (int it = 0; it < iters; ++it) {
        if constexpr (MODE == 13) {
#pragma unroll
            for (int r = 0; r < 4; ++r) acc3_mac<B>(a, x, y);
        } else {
#pragma unroll
            for (int r = 0; r < 2; ++r) { acc3_mac<B>(a, x, y); acc3_mac<B>(b, y, x); }
        }
#pragma unroll
        for (int i = 0; i < B; ++i) x[i] ^= a.E[i] + b.E[i];
    }
    uint32_t V[2 * B + 2], U[2 * B + 2];
    acc3_value<B>(V, a);
    acc3_value<B>(U, b);
#pragma unroll
    for (int j = 0; j < 2 * B + 2; ++j) fold ^= V[j] + U[j];
    __syncthreads();
    long long t1 = clock64();
    sink[blockIdx.x * blockDim.x + threadIdx.x] = fold;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

static void launch_acc(int mode, int sms, int iters, cudaStream_t st, uint32_t *sink, long long *cyc) {
    switch (mode) {
        case 9: k_bench_acc<9><<<sms, 768, 0, st>>>(iters, 12345u, sink, cyc); break;
        case 10: k_bench_acc<10><<<sms, 768, 0, st>>>(iters, 12345u, sink, cyc); break;
        case 11: k_bench_acc<11><<<sms, 768, 0, st>>>(iters, 12345u, sink, cyc); break;
        case 13: k_bench_ilp<13><<<sms, 256, 0, st>>>(iters, 12345u, sink, cyc); break;
        case 14: k_bench_ilp<14><<<sms, 256, 0, st>>>(iters, 12345u, sink, cyc); break;
        default: k_bench_acc<12><<<sms, 768, 0, st>>>(iters, 12345u, sink, cyc); break;
    }
}

extern "C" int mp_bench_imad(int mode, int iters, double *per_clk_per_sm, double *sm_mhz, void *stream) {
    if (mode < 0 || mode > 14 || iters <= 0 || !per_clk_per_sm) return MP_ERR_ARG;
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
    if (mode == 8) {
        k_bench_wide<<<sms, 512, 0, st>>>(1, 12345u, sink, cyc);   // warm-up
        cudaEventRecord(e0, st);
        k_bench_wide<<<sms, 512, 0, st>>>(iters, 12345u, sink, cyc);
    } else if (mode >= 9) {
        launch_acc(mode, sms, 1, st, sink, cyc);   // warm-up
        cudaEventRecord(e0, st);
        launch_acc(mode, sms, iters, st, sink, cyc);
    } else {
        k_bench<<<sms, threads, 0, st>>>(mode, 1, 12345u, sink, cyc);   // warm-up
        cudaEventRecord(e0, st);
        k_bench<<<sms, threads, 0, st>>>(mode, iters, 12345u, sink, cyc);
    }
    cudaEventRecord(e1, st);
    int rc = (cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess) ? MP_OK : MP_ERR_CUDA;
    if (rc == MP_OK) {
        std::vector<long long> c(sms);
        cudaMemcpy(c.data(), cyc, (size_t)sms * 8, cudaMemcpyDeviceToHost);
        std::sort(c.begin(), c.end());
        const double med = (double)c[sms / 2];
        // multiply-adds per thread: every mode is sized to 128 per iteration (mode 6: 256),
        // mode 7 runs on a quarter of the threads
        const double per_thread = (mode == 6 ? 256.0 : mode == 8 ? 200.0 : 128.0) * iters;
        const double active = (mode == 7 || mode >= 13) ? 256.0 : mode == 8 ? 512.0 : mode >= 9 ? 768.0 : (double)threads;
        *per_clk_per_sm = per_thread * active / med;
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
