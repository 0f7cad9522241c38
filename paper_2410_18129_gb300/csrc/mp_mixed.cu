// Mixed-size constant-time exponentiation in one persistent launch: job checks,
// workspace, tile numbering and the launch (the kernel is in mp_mixed.cuh).
#include "mp_mixed.cuh"

namespace mpg {

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
    if (red != MP_RED_TRUNCATED && red != MP_RED_FULL && red != MP_RED_CIOS) return MP_ERR_ARG;
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
    const cudaError_t e = red == MP_RED_TRUNCATED ? launch_mixed_red0(P, st)
                          : red == MP_RED_FULL    ? launch_mixed_red1(P, st)
                                                  : launch_mixed_red2(P, st);
    return e == cudaSuccess ? MP_OK : MP_ERR_CUDA;
}
