// Mixed-size constant-time exponentiation in one persistent launch.
//
// Instances of several sizes (each job = one Montgomery context and its bases,
// exponents and outputs) are cut into tiles of one block's worth of instances.
// Tiles are numbered job by job, the costliest job first, and every resident
// block pulls the next tile number from one atomic counter until none are left,
// so the large instances start first and the small ones fill the tail. A tile
// runs the same per-group exponentiation as the one-size kernel, with the group
// shape of its size class. Only sizes, shapes and tile numbers (public data)
// decide the control flow.
#include <cuda_runtime.h>
#include <algorithm>
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

// the persistent kernel's shape id for this context: the shape selected for its size
// class if the kernel has it, else another compiled shape of the same padded size
static int mix_shape_for(const mont_ctx *c, int *G) {
    int g = 0, m = 0;
    if (mp_tune_get(c->bits, &g, &m, nullptr, nullptr) != MP_OK) return -1;
    static const int GM[MIX_NSHAPES][2] = {{4, 4}, {4, 8}, {8, 4}, {8, 8}, {16, 4}, {8, 12}, {16, 6}, {16, 8}};
    int other = -1;
    for (int i = 0; i < MIX_NSHAPES; ++i) {
        if ((uint32_t)(GM[i][0] * GM[i][1]) != c->np) continue;
        if (GM[i][0] == g && GM[i][1] == m) {
            *G = g;
            return i;
        }
        if (other < 0) other = i;
    }
    if (other >= 0) *G = GM[other][0];
    return other;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static size_t job_table_bytes(const mp_modexp_job &j) {
    if (j.index) return 0;   // fixed-base job: resident tables
    const uint32_t w = j.window ? j.window : default_window(j.ctx->bits);
    return ((size_t)1 << w) * (size_t)j.ctx->np * j.ctx->batch * 4;
}

static size_t job_instances(const mp_modexp_job &j) { return j.index ? j.nreq : j.ctx->batch; }

template <int RED>
static cudaError_t launch_mixed(const MixArgs &P, cudaStream_t st) {
    static int grid = 0;   // resident blocks over the whole GPU, computed once per process
    if (!grid) {
        cudaError_t e = cudaFuncSetAttribute(k_modexp_mixed<RED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)MIX_SMEM);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per_sm = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_modexp_mixed<RED>, MIX_TPB, MIX_SMEM)) !=
            cudaSuccess)
            return e;
        grid = sms * (per_sm > 0 ? per_sm : 1);
    }
    const int blocks = std::min(grid, P.total > 0 ? P.total : 1);
    k_modexp_mixed<RED><<<blocks, MIX_TPB, MIX_SMEM, st>>>(P);
    return cudaGetLastError();
}

}  // namespace mpg

using namespace mpg;

static int check_jobs(const mp_modexp_job *jobs, int njobs) {
    if (!jobs || njobs <= 0) return MP_ERR_ARG;
    if (njobs > MIX_MAX_JOBS) return MP_ERR_SIZE;
    for (int i = 0; i < njobs; ++i) {
        const mp_modexp_job &j = jobs[i];
        if (!j.y || !j.ctx || (j.exp_bits > 0 && !j.exp)) return MP_ERR_ARG;
        if (j.index ? (!j.tables || j.nreq == 0 || j.window == 0) : !j.base) return MP_ERR_ARG;
        if (j.window > 6) return MP_ERR_SIZE;
        if (j.index && ((uintptr_t)j.tables & 15u)) return MP_ERR_ALIGN;
        int G = 0;
        if (mix_shape_for(j.ctx, &G) < 0) return MP_ERR_UNIMPLEMENTED;
        if (j.ctx->layout == MP_LAYOUT_INTERLEAVED &&
            ((((uintptr_t)j.y) | ((uintptr_t)j.base) | ((uintptr_t)j.exp)) & 15u))
            return MP_ERR_ALIGN;
    }
    return MP_OK;
}

extern "C" size_t modexp_mixed_workspace_bytes(const mp_modexp_job *jobs, int njobs) {
    if (check_jobs(jobs, njobs) != MP_OK) return 0;
    size_t total = 256;   // tile counter
    for (int i = 0; i < njobs; ++i) total += align256(job_table_bytes(jobs[i]));
    return total;
}

extern "C" int modexp_consttime_mixed(const mp_modexp_job *jobs, int njobs, mp_red red, void *workspace,
                                      size_t workspace_bytes, void *stream) {
    int rc = check_jobs(jobs, njobs);
    if (rc != MP_OK) return rc;
    if (red == MP_RED_CIOS) return MP_ERR_UNIMPLEMENTED;   // the persistent kernel carries Alg. 5/6 only
    if (red != MP_RED_TRUNCATED && red != MP_RED_FULL) return MP_ERR_ARG;
    if (!workspace || ((uintptr_t)workspace & 255u)) return workspace ? MP_ERR_ALIGN : MP_ERR_ARG;
    if (workspace_bytes < modexp_mixed_workspace_bytes(jobs, njobs)) return MP_ERR_NOMEM;
    // costliest job first: cost per instance ~ words^2 * exponent bits
    int order[MIX_MAX_JOBS];
    for (int i = 0; i < njobs; ++i) order[i] = i;
    std::stable_sort(order, order + njobs, [&](int x, int y) {
        const double cx = (double)jobs[x].ctx->np * jobs[x].ctx->np * (jobs[x].exp_bits + 64);
        const double cy = (double)jobs[y].ctx->np * jobs[y].ctx->np * (jobs[y].exp_bits + 64);
        return cx > cy;
    });
    MixArgs P{};
    char *ws = static_cast<char *>(workspace);
    P.counter = reinterpret_cast<unsigned *>(ws);
    size_t off = 256;
    int tile = 0;
    for (int r = 0; r < njobs; ++r) {
        const mp_modexp_job &j = jobs[order[r]];
        MixJob &J = P.job[r];
        ctx_args(J.A, j.ctx);
        J.A.out = j.y;
        J.A.a = j.base;
        J.A.e = j.exp;
        J.A.ebits = (int)j.exp_bits;
        J.A.ne = j.exp_bits ? (int)((j.exp_bits + 31) / 32) : 1;
        J.A.window = (int)(j.window ? j.window : default_window(j.ctx->bits));
        J.A.red = (int)red;
        if (j.index) {   // fixed-base requests on resident tables
            J.A.index = j.index;
            J.A.batch = j.nreq;
            J.A.table = const_cast<uint32_t *>(reinterpret_cast<const uint32_t *>(j.tables));
            J.A.mode = 2;
        } else {
            J.A.table = reinterpret_cast<uint32_t *>(ws + off);
            off += align256(job_table_bytes(j));
        }
        int G = 0;
        J.shape = mix_shape_for(j.ctx, &G);
        const int gpb = MIX_TPB / G;
        J.tile0 = tile;
        tile += (int)((job_instances(j) + gpb - 1) / gpb);
    }
    P.njobs = njobs;
    P.total = tile;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(P.counter, 0, sizeof(unsigned), st) != cudaSuccess) return MP_ERR_CUDA;
    const cudaError_t e = red == MP_RED_TRUNCATED ? launch_mixed<0>(P, st) : launch_mixed<1>(P, st);
    return e == cudaSuccess ? MP_OK : MP_ERR_CUDA;
}
