// Mixed-size constant-time exponentiation: job checks, workspace, and one launch per job of
// its size class's own kernel, forked onto parallel streams costliest job first and joined
// back to the caller's stream.
//
// Each size class has its own block shape (threads per instance, instances per block, shared
// memory per block). A single kernel for every size would have to size its blocks for the
// largest class and lose occupancy on the others; instead every job runs the kernel that
// modexp_consttime would run for it, at full occupancy. The jobs are independent, so they
// run on separate streams: the costliest job's blocks are issued first and the GPU fills the
// last partial wave of one job with blocks of the next. The fork (an event recorded on the
// caller's stream that every job stream waits for) and the join (an event per job that the
// caller's stream waits for) are stream operations, so the whole call can be captured in a
// CUDA graph together with its input and result copies.
#include <cuda_runtime.h>
#include <algorithm>
#include <mutex>
#include "mp_internal.h"

namespace mpg {

constexpr int MIX_MAX_JOBS = 16;
constexpr int MIX_STREAMS = 8;
constexpr int MIX_MAX_DEVICES = 64;

// Streams and events of the fork/join, created once per device with that device current
// (non-blocking streams: they synchronise with the caller only through the events).
struct MixPool {
    bool ready = false;
    cudaStream_t s[MIX_STREAMS];
    cudaEvent_t fork;
    cudaEvent_t join[MIX_MAX_JOBS];
    int next = 0;   // round robin over the streams across calls
};
static MixPool g_pool[MIX_MAX_DEVICES];
static std::mutex g_pool_mu;   // guards g_pool and the record/wait sequence of a call

static cudaError_t pool_init(MixPool &p) {
    if (p.ready) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < MIX_STREAMS && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&p.s[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming);
    for (int i = 0; i < MIX_MAX_JOBS && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&p.join[i], cudaEventDisableTiming);
    if (e == cudaSuccess) p.ready = true;
    return e;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// fixed-base job: resident tables; otherwise one table per request (per context instance
// without routing)
static bool job_fixed(const mp_modexp_job &j) { return j.index && j.tables; }

static size_t job_instances(const mp_modexp_job &j) { return j.index ? j.nreq : j.ctx->batch; }

static size_t job_table_bytes(const mp_modexp_job &j) {
    if (job_fixed(j)) return 0;
    const uint32_t w = j.window ? j.window : default_window(j.ctx->bits);
    return ((size_t)1 << w) * (size_t)j.ctx->np * job_instances(j) * 4;
}

}  // namespace mpg

using namespace mpg;

static int check_jobs(const mp_modexp_job *jobs, int njobs) {
    if (!jobs || njobs <= 0) return MP_ERR_ARG;
    if (njobs > MIX_MAX_JOBS) return MP_ERR_SIZE;
    for (int i = 0; i < njobs; ++i) {
        const mp_modexp_job &j = jobs[i];
        if (!j.y || !j.ctx || (j.exp_bits > 0 && !j.exp)) return MP_ERR_ARG;
        if (j.index ? (j.nreq == 0 || (j.tables ? j.window == 0 : !j.base)) : !j.base) return MP_ERR_ARG;
        if (j.window > 6) return MP_ERR_SIZE;
        if (j.index && ((uintptr_t)j.tables & 15u)) return MP_ERR_ALIGN;
        if (j.ctx->layout == MP_LAYOUT_INTERLEAVED &&
            ((((uintptr_t)j.y) | ((uintptr_t)j.base) | ((uintptr_t)j.exp)) & 15u))
            return MP_ERR_ALIGN;
    }
    return MP_OK;
}

extern "C" size_t modexp_mixed_workspace_bytes(const mp_modexp_job *jobs, int njobs) {
    if (check_jobs(jobs, njobs) != MP_OK) return 0;
    size_t total = 256;
    for (int i = 0; i < njobs; ++i) total += align256(job_table_bytes(jobs[i]));
    return total;
}

extern "C" int modexp_consttime_mixed(const mp_modexp_job *jobs, int njobs, mp_red red, void *workspace,
                                      size_t workspace_bytes, void *stream) {
    int rc = check_jobs(jobs, njobs);
    if (rc != MP_OK) return rc;
    if (red != MP_RED_TRUNCATED && red != MP_RED_FULL && red != MP_RED_CIOS) return MP_ERR_ARG;
    if (!workspace || ((uintptr_t)workspace & 255u)) return workspace ? MP_ERR_ALIGN : MP_ERR_ARG;
    if (workspace_bytes < modexp_mixed_workspace_bytes(jobs, njobs)) return MP_ERR_NOMEM;
    // costliest job first: cost ~ instances * words^2 * exponent bits
    int order[MIX_MAX_JOBS];
    for (int i = 0; i < njobs; ++i) order[i] = i;
    std::stable_sort(order, order + njobs, [&](int x, int y) {
        const auto cost = [&](const mp_modexp_job &j) {
            return (double)job_instances(j) * j.ctx->np * j.ctx->np * (j.exp_bits + 64);
        };
        return cost(jobs[x]) > cost(jobs[y]);
    });
    // argument blocks and kernels of every job (host checks before any launch)
    KArgs args[MIX_MAX_JOBS];
    const ShapeOps *ops[MIX_MAX_JOBS];
    char *ws = static_cast<char *>(workspace);
    size_t off = 256;
    for (int r = 0; r < njobs; ++r) {
        const mp_modexp_job &j = jobs[order[r]];
        ops[r] = shape_for_red_np(j.ctx->np, (int)red);
        if (!ops[r]) return MP_ERR_UNIMPLEMENTED;
        KArgs &A = args[r];
        A = KArgs{};
        ctx_args(A, j.ctx);
        A.out = j.y;
        A.a = j.base;
        A.e = j.exp;
        A.ebits = (int)j.exp_bits;
        A.ne = j.exp_bits ? (int)((j.exp_bits + 31) / 32) : 1;
        A.window = (int)(j.window ? j.window : default_window(j.ctx->bits));
        A.red = (int)red;
        if (j.index) {   // requests routed to context instances
            A.index = j.index;
            A.batch = j.nreq;
        }
        if (job_fixed(j)) {   // fixed bases: resident tables
            A.table = const_cast<uint32_t *>(reinterpret_cast<const uint32_t *>(j.tables));
            A.mode = 2;
        } else {              // own bases: tables built in the workspace, one per request
            A.table = reinterpret_cast<uint32_t *>(ws + off);
            off += align256(job_table_bytes(j));
        }
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (njobs == 1) return ops[0]->modexp(args[0], st) == cudaSuccess ? MP_OK : MP_ERR_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MIX_MAX_DEVICES) return MP_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    MixPool &p = g_pool[dev];
    if (pool_init(p) != cudaSuccess) return MP_ERR_CUDA;
    cudaError_t e = cudaEventRecord(p.fork, st);
    for (int r = 0; r < njobs && e == cudaSuccess; ++r) {
        cudaStream_t js = p.s[(p.next + r) % MIX_STREAMS];
        e = cudaStreamWaitEvent(js, p.fork, 0);
        if (e == cudaSuccess) e = ops[r]->modexp(args[r], js);
        if (e == cudaSuccess) e = cudaEventRecord(p.join[r], js);
    }
    // join every forked stream (also after a failure, so no stream is left out of a capture)
    for (int r = 0; r < njobs; ++r) {
        const cudaError_t w = cudaStreamWaitEvent(st, p.join[r], 0);
        if (e == cudaSuccess) e = w;
    }
    p.next = (p.next + njobs) % MIX_STREAMS;
    return e == cudaSuccess ? MP_OK : MP_ERR_CUDA;
}
