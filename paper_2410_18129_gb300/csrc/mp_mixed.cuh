// Mixed-size constant-time exponentiation in one persistent launch: the kernel.
//
// Instances of several sizes (each job = one Montgomery context and its bases,
// exponents and outputs) are cut into tiles of one block's worth of instances.
// Tiles are numbered job by job, the costliest job first, and every resident
// block pulls the next tile number from one atomic counter until none are left,
// so the large instances start first and the small ones fill the tail. A tile
// runs the same per-group exponentiation as the one-size kernel, with the group
// shape of its size class. Only sizes, shapes and tile numbers (public data)
// decide the control flow. One translation unit per reduction instantiates it.
#pragma once
#include <cuda_runtime.h>
#include <algorithm>
#include <atomic>
#include "mp_internal.h"

namespace mpg {

constexpr int MIX_TPB = 256;
constexpr int MIX_MAX_JOBS = 16;

// every compiled group shape of the sizes up to 4096 bits; a job runs with the shape
// currently selected for its size class (see mp_tune_set)
using MixS0 = Shape<4, 4>;    //  512 bits
using MixS1 = Shape<4, 8>;    // 1024 bits
using MixS2 = Shape<8, 4>;    // 1024 bits
using MixS3 = Shape<8, 8>;    // 2048 bits
using MixS4 = Shape<16, 4>;   // 2048 bits
using MixS5 = Shape<8, 12>;   // 3072 bits
using MixS6 = Shape<16, 6>;   // 3072 bits
using MixS7 = Shape<16, 8>;   // 4096 bits
constexpr int MIX_NSHAPES = 8;

template <class S>
constexpr size_t mix_smem() { return (size_t)(MIX_TPB / S::G) * S::WORDS * 4; }
constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t MIX_SMEM =
    cmax(cmax(cmax(mix_smem<MixS0>(), mix_smem<MixS1>()), cmax(mix_smem<MixS2>(), mix_smem<MixS3>())),
         cmax(cmax(mix_smem<MixS4>(), mix_smem<MixS5>()), cmax(mix_smem<MixS6>(), mix_smem<MixS7>())));

struct MixJob {
    KArgs A;
    int shape;   // 0..7: MixS0..MixS7
    int tile0;   // first tile number of this job
};

struct MixArgs {
    MixJob job[MIX_MAX_JOBS];
    int njobs;
    int total;           // tiles over all jobs
    unsigned *counter;   // next tile number (zeroed before the launch)
};

template <class S, int RED>
MPG_DI void mix_tile(const KArgs &A, int tile, uint32_t *smem) {
    Grp<S> g = make_group<S>(smem);
    const size_t k = (size_t)tile * (MIX_TPB / S::G) + threadIdx.x / S::G;
    modexp_group<S, RED>(g, A, k);
}

template <int RED>
__global__ void __launch_bounds__(MIX_TPB, 2) k_modexp_mixed(const __grid_constant__ MixArgs P) {
    extern __shared__ uint4 smem4[];
    uint32_t *smem = reinterpret_cast<uint32_t *>(smem4);
    __shared__ int s_tile;
    for (;;) {
        __syncthreads();   // the previous tile is finished in every warp
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(P.counter, 1u);
        __syncthreads();
        const int tile = s_tile;
        if (tile >= P.total) break;
        int j = 0;
        while (j + 1 < P.njobs && tile >= P.job[j + 1].tile0) ++j;
        const MixJob &J = P.job[j];
        const int local = tile - J.tile0;
        switch (J.shape) {
            case 0: mix_tile<MixS0, RED>(J.A, local, smem); break;
            case 1: mix_tile<MixS1, RED>(J.A, local, smem); break;
            case 2: mix_tile<MixS2, RED>(J.A, local, smem); break;
            case 3: mix_tile<MixS3, RED>(J.A, local, smem); break;
            case 4: mix_tile<MixS4, RED>(J.A, local, smem); break;
            case 5: mix_tile<MixS5, RED>(J.A, local, smem); break;
            case 6: mix_tile<MixS6, RED>(J.A, local, smem); break;
            default: mix_tile<MixS7, RED>(J.A, local, smem); break;
        }
    }
}

template <int RED>
cudaError_t launch_mixed(const MixArgs &P, cudaStream_t st) {
    // resident blocks over the whole GPU, computed once per device (with its attribute call)
    static std::atomic<int> grids[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int grid = (dev >= 0 && dev < 64) ? grids[dev].load(std::memory_order_acquire) : 0;
    if (!grid) {
        e = cudaFuncSetAttribute(k_modexp_mixed<RED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MIX_SMEM);
        if (e != cudaSuccess) return e;
        int sms = 0, per_sm = 0;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_modexp_mixed<RED>, MIX_TPB, MIX_SMEM)) !=
            cudaSuccess)
            return e;
        grid = sms * (per_sm > 0 ? per_sm : 1);
        if (dev >= 0 && dev < 64) grids[dev].store(grid, std::memory_order_release);
    }
    const int blocks = std::min(grid, P.total > 0 ? P.total : 1);
    k_modexp_mixed<RED><<<blocks, MIX_TPB, MIX_SMEM, st>>>(P);
    return cudaGetLastError();
}

// one instantiation per reduction (mp_mixed_red*.cu)
cudaError_t launch_mixed_red0(const MixArgs &P, cudaStream_t st);
cudaError_t launch_mixed_red1(const MixArgs &P, cudaStream_t st);
cudaError_t launch_mixed_red2(const MixArgs &P, cudaStream_t st);

}  // namespace mpg
