// C ABI of the library (include/mpgpu.h): argument checks, shape dispatch,
// Montgomery-context construction and the layout conversion kernel.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <atomic>
#include <cstring>
#include <mutex>
#include <new>
#include "mp_internal.h"

namespace mpg {
ShapeOps shape_ops_2_4();
ShapeOps shape_ops_4_4();
ShapeOps shape_ops_4_8();
ShapeOps shape_ops_8_4();
ShapeOps shape_ops_8_8();
ShapeOps shape_ops_16_4();
ShapeOps shape_ops_8_12();
ShapeOps shape_ops_16_6();
ShapeOps shape_ops_8_16();
ShapeOps shape_ops_16_8();
ShapeOps shape_ops_8_18();
ShapeOps shape_ops_8_8_w();
cudaError_t kara2_128(const KArgs &, cudaStream_t);
cudaError_t kara2_144(const KArgs &, cudaStream_t);
unsigned long long dbg_take_kara2();
ShapeOps tkara_ops_16();
ShapeOps tkara_ops_32();
ShapeOps tkara_ops_64();
ShapeOps tkara_ops_96();
ShapeOps tkara_ops_128();
}  // namespace mpg

using namespace mpg;

static constexpr uint32_t MAX_NP = 144;   // largest padded size: 8 threads x 18 words
static constexpr uint32_t MAX_BITS = 32 * MAX_NP;
// MP_ALGO_AUTO switch-over for products: measured on GB300, schoolbook wins at every size
// (M products/s at a batch of 65536, schoolbook vs one Karatsuba level; role-swapped kernels:
// 1024 bits mul 3826 / 3035, sqr 4980 / 3454; 2048 bits 1429 / 1218, 1932 / 1504; 3072 bits
// 762 / 661, 1175 / 907; 4096 bits 470 / 464, 671 / 662; 4108 and 4154 bits, lane-mapped
// schoolbook and role-swapped Karatsuba: 305 / 300, 458 / 448), so AUTO never picks Karatsuba
// unless mp_tune_set sets a switch-over
static constexpr uint32_t KARATSUBA_FROM_BITS = 0xffffffffu;

// Size classes: one per padded size NP. Each class has one or more compiled group
// shapes (threads per instance x words per thread); the first is the default and
// mp_tune_set may select another, together with the default window width.
struct SizeClass {
    uint32_t np;
    int nshapes;
    ShapeOps shapes[3];
    int chosen;          // index into shapes
    uint32_t window;     // default window for modexp (0: built-in rule)
    uint32_t kara_from;  // AUTO products use Karatsuba from this many bits (0: built-in rule)
    cudaError_t (*kara2)(const KArgs &, cudaStream_t);   // two-level Karatsuba products, or null
    ShapeOps tk;         // Montgomery products in the truncated Karatsuba form (mont/modexp null if absent)
    uint32_t mont_kara_from;   // AUTO Montgomery products and exponentiations of the truncated reduction use
                               // the Karatsuba form from this many bits (0: never)
    int table_shared;          // modexp_consttime keeps the window tables in shared memory where they fit
};
static SizeClass g_classes[7];
static std::once_flag g_classes_once;

static void fill_classes() {
    g_classes[0] = SizeClass{8, 1, {shape_ops_2_4()}, 0, 0, 0};
    g_classes[1] = SizeClass{16, 1, {shape_ops_4_4()}, 0, 0, 0};
    g_classes[2] = SizeClass{32, 2, {shape_ops_4_8(), shape_ops_8_4()}, 0, 0, 0};
    g_classes[3] = SizeClass{64, 3, {shape_ops_8_8(), shape_ops_16_4(), shape_ops_8_8_w()}, 0, 0, 0};
    g_classes[4] = SizeClass{96, 2, {shape_ops_8_12(), shape_ops_16_6()}, 0, 0, 0};
    g_classes[5] = SizeClass{128, 2, {shape_ops_16_8(), shape_ops_8_16()}, 0, 0, 0, kara2_128};   // 16x8 faster
    g_classes[6] = SizeClass{144, 1, {shape_ops_8_18()}, 0, 0, 0, kara2_144};
    g_classes[1].tk = tkara_ops_16();    // the 256-bit class has no half shape (2 x 2 words)
    g_classes[2].tk = tkara_ops_32();
    g_classes[3].tk = tkara_ops_64();
    g_classes[4].tk = tkara_ops_96();
    g_classes[5].tk = tkara_ops_128();   // the 4608-bit class neither (8 x 9 has odd half blocks)
}

static void init_classes() { std::call_once(g_classes_once, fill_classes); }

static SizeClass *class_for(uint32_t n) {
    init_classes();
    for (auto &c : g_classes)
        if (c.np >= n) return &c;
    return nullptr;
}

// the selected shape for operands of n words
static const ShapeOps *shape_for(uint32_t n) {
    SizeClass *c = class_for(n);
    return c ? &c->shapes[c->chosen] : nullptr;
}

// the shape for a Montgomery product with reduction `red`: CIOS passes a word between the
// threads of an instance at every step, so it runs on a lane-mapped shape of the class
static const ShapeOps *shape_for_red(uint32_t n, int red) {
    SizeClass *c = class_for(n);
    if (!c) return nullptr;
    if (red == MP_RED_CIOS && c->shapes[c->chosen].G < 0)
        for (int i = 0; i < c->nshapes; ++i)
            if (c->shapes[i].G > 0) return &c->shapes[i];
    return &c->shapes[c->chosen];
}



static inline uint32_t words_for(uint32_t bits) { return (bits + 31u) / 32u; }
static inline size_t api_array_words(mp_layout layout, size_t batch, uint32_t words) {
    return layout == MP_LAYOUT_INTERLEAVED ? (size_t)((words + 3u) / 4u) * 4u * batch : (size_t)words * batch;
}
static inline bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }
static inline cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }

extern "C" const char *mp_strerror(int st) {
    switch (st) {
        case MP_OK: return "ok";
        case MP_ERR_ARG: return "invalid argument";
        case MP_ERR_SIZE: return "operand size or window out of range";
        case MP_ERR_EVEN_MODULUS: return "even modulus";
        case MP_ERR_ALIGN: return "pointer not 16-byte aligned";
        case MP_ERR_CUDA: return "CUDA error";
        case MP_ERR_NOMEM: return "out of device memory or workspace too small";
        case MP_ERR_UNIMPLEMENTED: return "not implemented";
        default: return "unknown status";
    }
}

extern "C" uint32_t mp_max_bits(void) { return MAX_BITS; }
extern "C" const char *mp_version(void) { return "mpgpu 0.1 (sm_103a)"; }

static int check_layout(mp_layout l) { return (l == MP_LAYOUT_INSTANCE_MAJOR || l == MP_LAYOUT_INTERLEAVED) ? MP_OK : MP_ERR_ARG; }

static int cuda_status(cudaError_t e) { return e == cudaSuccess ? MP_OK : MP_ERR_CUDA; }

// ------------------------------------------------------------------ layout conversion

__global__ void k_convert(uint32_t *dst, int dl, const uint32_t *src, int sl, size_t batch, int words) {
    // destination positions, padding words of an interleaved destination included
    const size_t total = (dl == LAYOUT_IL) ? (size_t)((words + 3) / 4) * 4 * batch : batch * (size_t)words;
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (size_t)gridDim.x * blockDim.x) {
        // enumerate in destination order so that the stores are coalesced
        size_t k;
        int i;
        if (dl == LAYOUT_IM) { k = x / (size_t)words; i = (int)(x % (size_t)words); }
        else {
            const size_t chunk = x / (4 * batch), r = x % (4 * batch);
            k = r / 4;
            i = (int)(chunk * 4 + r % 4);
            if (i >= words) continue;
        }
        dst[widx(dl, k, i, words, batch)] = src[widx(sl, k, i, words, batch)];
    }
}

static int launch_convert(uint32_t *dst, int dl, const uint32_t *src, int sl, size_t batch, int words, cudaStream_t st) {
    size_t total = (dl == LAYOUT_IL) ? (size_t)((words + 3) / 4) * 4 * batch : (size_t)words * batch;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MP_ERR_CUDA;
    const size_t cap = (size_t)(sms > 0 ? sms : 1) * 32u;   // grid-stride loop: 32 blocks of 256 per SM at most
    size_t blocks = (total + 255) / 256;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) blocks = 1;
    k_convert<<<(unsigned)blocks, 256, 0, st>>>(dst, dl, src, sl, batch, words);
    return cuda_status(cudaGetLastError());
}

extern "C" int mp_convert(uint32_t *dst, mp_layout dst_layout, const uint32_t *src, mp_layout src_layout,
                          size_t batch, uint32_t words, void *stream) {
    if (!dst || !src || batch == 0 || words == 0) return MP_ERR_ARG;
    if (check_layout(dst_layout) || check_layout(src_layout)) return MP_ERR_ARG;
    if ((dst_layout == MP_LAYOUT_INTERLEAVED && !aligned16(dst)) ||
        (src_layout == MP_LAYOUT_INTERLEAVED && !aligned16(src)))
        return MP_ERR_ALIGN;
    if (dst_layout == src_layout)
        return cuda_status(cudaMemcpyAsync(dst, src, api_array_words(dst_layout, batch, words) * 4,
                                           cudaMemcpyDeviceToDevice, S(stream)));
    return launch_convert(dst, (int)dst_layout, src, (int)src_layout, batch, (int)words, S(stream));
}

// ------------------------------------------------------------------ products

static int check_common(size_t batch, uint32_t bits, mp_layout layout, mp_algo algo) {
    if (batch == 0) return MP_ERR_ARG;
    if (check_layout(layout)) return MP_ERR_ARG;
    if (algo != MP_ALGO_AUTO && algo != MP_ALGO_SCHOOLBOOK && algo != MP_ALGO_KARATSUBA &&
        algo != MP_ALGO_KARATSUBA2)
        return MP_ERR_ARG;
    if (bits == 0 || bits > MAX_BITS) return MP_ERR_SIZE;
    return MP_OK;
}

static int product(uint32_t *c, const uint32_t *a, const uint32_t *b, size_t batch, uint32_t bits,
                   mp_layout layout, mp_algo algo, bool square, void *stream) {
    if (!c || !a || (!square && !b)) return MP_ERR_ARG;
    int st = check_common(batch, bits, layout, algo);
    if (st) return st;
    if (layout == MP_LAYOUT_INTERLEAVED && (!aligned16(c) || !aligned16(a) || (!square && !aligned16(b))))
        return MP_ERR_ALIGN;
    const uint32_t n = words_for(bits);
    const ShapeOps *sh = shape_for(n);
    if (!sh) return MP_ERR_SIZE;
    KArgs A{};
    A.out = c; A.a = a; A.b = square ? a : b;
    A.batch = batch; A.cbatch = batch; A.n = (int)n; A.layout = (int)layout; A.square = square ? 1 : 0;
    const SizeClass *cls = class_for(n);
    if (algo == MP_ALGO_KARATSUBA2)
        return cls->kara2 ? cuda_status(cls->kara2(A, S(stream))) : MP_ERR_UNIMPLEMENTED;
    const uint32_t kfrom = cls->kara_from ? cls->kara_from : KARATSUBA_FROM_BITS;
    bool kara = algo == MP_ALGO_KARATSUBA || (algo == MP_ALGO_AUTO && bits >= kfrom);
    const ShapeOps *ksh = sh->kara ? sh : nullptr;   // any shape of the class with a Karatsuba kernel
    for (int i = 0; i < cls->nshapes && !ksh; ++i)
        if (cls->shapes[i].kara) ksh = &cls->shapes[i];
    if (kara && !ksh) {
        if (algo == MP_ALGO_KARATSUBA) return MP_ERR_UNIMPLEMENTED;
        kara = false;
    }
    return cuda_status(kara ? ksh->kara(A, S(stream)) : sh->mul(A, S(stream)));
}

extern "C" int mp_mul(uint32_t *c, const uint32_t *a, const uint32_t *b, size_t batch, uint32_t bits,
                      mp_layout layout, mp_algo algo, void *stream) {
    return product(c, a, b, batch, bits, layout, algo, false, stream);
}

extern "C" int mp_sqr(uint32_t *c, const uint32_t *a, size_t batch, uint32_t bits, mp_layout layout,
                      mp_algo algo, void *stream) {
    return product(c, a, nullptr, batch, bits, layout, algo, true, stream);
}

// ------------------------------------------------------------------ Montgomery context

// x <- 2x mod N (x < N), np words, select without a branch
__device__ void dbl_mod(uint32_t *x, const uint32_t *N, int np) {
    uint32_t carry = 0;
    for (int i = 0; i < np; ++i) {
        const uint32_t v = x[i];
        x[i] = (v << 1) | carry;
        carry = v >> 31;
    }
    uint32_t d[MAX_NP];
    uint32_t borrow = 0;
    for (int i = 0; i < np; ++i) {
        const uint64_t t = (uint64_t)x[i] - N[i] - borrow;
        d[i] = (uint32_t)t;
        borrow = (uint32_t)(t >> 63);
    }
    const uint32_t m = 0u - (carry | (borrow ^ 1u));
    for (int i = 0; i < np; ++i) x[i] = (d[i] & m) | (x[i] & ~m);
}

// One thread per modulus: N' by word-level Hensel lifting, powers of two mod N by
// modular doubling. Not on the hot path (runs once per modulus).
__global__ void k_ctx_init(const uint32_t *Napi, int layout, size_t batch, int n, int np, uint32_t *N,
                           uint32_t *NI, uint32_t *R1, uint32_t *R2, uint32_t *K, uint32_t *NI_api,
                           uint32_t *R1_api, uint32_t *R2_api, uint32_t *N_api, unsigned long long *bad) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= batch) return;
    uint32_t nn[MAX_NP], x[MAX_NP], p[MAX_NP], r1[MAX_NP];
    for (int i = 0; i < np; ++i) nn[i] = (i < n) ? Napi[widx(layout, k, i, n, batch)] : 0u;
    for (int i = 0; i < n; ++i) N_api[widx(layout, k, i, n, batch)] = nn[i];
    if ((nn[0] & 1u) == 0u) {
        atomicMin(bad, (unsigned long long)k);
        return;
    }
    // 32-bit inverse of N0 by Newton's iteration y <- y (2 - N0 y): 3, 6, 12, 24, 48 bits
    uint32_t y = nn[0];
    for (int it = 0; it < 4; ++it) y *= 2u - nn[0] * y;
    const uint32_t n0p = 0u - y;   // -N0^{-1} mod 2^32
    // word-level lifting: keep P = N*x + 1 mod W^np; x_i = P_i * n0p clears word i
    for (int i = 0; i < np; ++i) { p[i] = 0u; x[i] = 0u; }
    p[0] = 1u;
    for (int i = 0; i < np; ++i) {
        const uint32_t xi = p[i] * n0p;
        x[i] = xi;
        uint64_t c = 0;
        for (int j = 0; i + j < np; ++j) {
            c += (uint64_t)xi * nn[j] + p[i + j];
            p[i + j] = (uint32_t)c;
            c >>= 32;
        }
    }
    auto put_il = [&](uint32_t *dst, const uint32_t *src) {
        for (int i = 0; i < np; ++i) dst[widx(LAYOUT_IL, k, i, np, batch)] = src[i];
    };
    auto put_api = [&](uint32_t *dst, const uint32_t *src) {
        for (int i = 0; i < n; ++i) dst[widx(layout, k, i, n, batch)] = src[i];
    };
    put_il(N, nn);
    put_il(NI, x);
    put_api(NI_api, x);   // (-N)^-1 mod W^n is the low n words of (-N)^-1 mod W^np
    // powers of two: start at 1 and double
    for (int i = 0; i < np; ++i) p[i] = 0u;
    p[0] = 1u;
    for (int d = 0; d < 32 * n; ++d) dbl_mod(p, nn, np);
    put_api(R1_api, p);                               // W^n mod N
    for (int i = 0; i < np; ++i) r1[i] = p[i];
    for (int d = 0; d < 32 * n; ++d) dbl_mod(r1, nn, np);
    put_api(R2_api, r1);                              // W^2n mod N
    for (int d = 0; d < 32 * (np - n); ++d) dbl_mod(p, nn, np);
    put_il(R1, p);                                    // W^np mod N
    for (int i = 0; i < np; ++i) r1[i] = p[i];
    for (int d = 0; d < 32 * (np - n); ++d) dbl_mod(r1, nn, np);
    put_il(K, r1);                                    // W^(2np-n) mod N
    for (int d = 0; d < 32 * np; ++d) dbl_mod(p, nn, np);
    put_il(R2, p);                                    // W^2np mod N
}

extern "C" int mont_ctx_init(mont_ctx **out, const uint32_t *N, size_t batch, uint32_t bits, mp_layout layout,
                             size_t *bad_index, void *stream) {
    if (!out || !N || batch == 0) return MP_ERR_ARG;
    *out = nullptr;
    if (check_layout(layout)) return MP_ERR_ARG;
    if (bits < 2 || bits > MAX_BITS) return MP_ERR_SIZE;
    if (layout == MP_LAYOUT_INTERLEAVED && !aligned16(N)) return MP_ERR_ALIGN;
    const uint32_t n = words_for(bits);
    const ShapeOps *sh = shape_for(n);
    if (!sh) return MP_ERR_SIZE;
    mont_ctx *c = new (std::nothrow) mont_ctx{};
    if (!c) return MP_ERR_NOMEM;
    c->batch = batch; c->bits = bits; c->n = n; c->np = (uint32_t)sh->NP; c->layout = layout;
    c->stream = S(stream);
    c->api_words = api_array_words(layout, batch, n);
    const size_t internal = (size_t)c->np * batch;
    const size_t total = 5 * internal + 4 * c->api_words + 4;   // +4: the error word (8 bytes, kept aligned)
    if (cudaMallocAsync(&c->mem, total * 4, S(stream)) != cudaSuccess) {
        delete c;
        cudaGetLastError();
        return MP_ERR_NOMEM;
    }
    uint32_t *p = c->mem;
    c->N = p; p += internal;
    c->NI = p; p += internal;
    c->R1 = p; p += internal;
    c->R2 = p; p += internal;
    c->K = p; p += internal;
    c->NI_api = p; p += c->api_words;
    c->R1_api = p; p += c->api_words;
    c->R2_api = p; p += c->api_words;
    c->N_api = p; p += c->api_words;
    unsigned long long *bad = reinterpret_cast<unsigned long long *>(p);
    cudaStream_t st = S(stream);
    int rc = MP_OK;
    const unsigned long long none = ~0ull;
    unsigned long long first = none;
    do {
        if (cudaMemcpyAsync(bad, &none, 8, cudaMemcpyHostToDevice, st) != cudaSuccess) { rc = MP_ERR_CUDA; break; }
        if (cudaMemsetAsync(c->mem, 0, 5 * internal * 4, st) != cudaSuccess) { rc = MP_ERR_CUDA; break; }
        const unsigned blocks = (unsigned)((batch + 127) / 128);
        k_ctx_init<<<blocks, 128, 0, st>>>(N, (int)layout, batch, (int)n, (int)c->np, c->N, c->NI, c->R1, c->R2,
                                           c->K, c->NI_api, c->R1_api, c->R2_api, c->N_api, bad);
        if (cudaGetLastError() != cudaSuccess) { rc = MP_ERR_CUDA; break; }
        if (cudaMemcpyAsync(&first, bad, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) { rc = MP_ERR_CUDA; break; }
        if (cudaStreamSynchronize(st) != cudaSuccess) { rc = MP_ERR_CUDA; break; }
        if (first != none) {
            if (bad_index) *bad_index = (size_t)first;
            rc = MP_ERR_EVEN_MODULUS;
        }
    } while (0);
    if (rc != MP_OK) {
        cudaFreeAsync(c->mem, st);
        delete c;
        return rc;
    }
    *out = c;
    return MP_OK;
}

extern "C" int mont_ctx_free(mont_ctx *c) {
    if (!c) return MP_OK;
    // stream-ordered: the memory goes back after everything already queued on the context's
    // stream; no other stream or host thread waits
    const cudaError_t e = cudaFreeAsync(c->mem, c->stream);
    delete c;
    return e == cudaSuccess ? MP_OK : MP_ERR_CUDA;
}

extern "C" int mont_ctx_info(const mont_ctx *c, size_t *batch, uint32_t *bits, mp_layout *layout) {
    if (!c) return MP_ERR_ARG;
    if (batch) *batch = c->batch;
    if (bits) *bits = c->bits;
    if (layout) *layout = c->layout;
    return MP_OK;
}

extern "C" int mont_ctx_export(const mont_ctx *c, int which, uint32_t *dst, void *stream) {
    if (!c || !dst) return MP_ERR_ARG;
    const uint32_t *src = which == 0 ? c->NI_api : which == 1 ? c->R1_api : which == 2 ? c->R2_api
                        : which == 3 ? c->N_api : nullptr;
    if (!src) return MP_ERR_ARG;
    if (c->layout == MP_LAYOUT_INTERLEAVED && !aligned16(dst)) return MP_ERR_ALIGN;
    return cuda_status(cudaMemcpyAsync(dst, src, c->api_words * 4, cudaMemcpyDeviceToDevice, S(stream)));
}

// ------------------------------------------------------------------ Montgomery products

static void fill_ctx_args(KArgs &A, const mont_ctx *c) {
    A.N = c->N; A.NI = c->NI; A.R1 = c->R1; A.R2 = c->R2; A.K = c->K;
    A.batch = c->batch; A.cbatch = c->batch; A.n = (int)c->n; A.layout = (int)c->layout;
    A.correct = (c->n != c->np) ? 1 : 0;
    A.index = nullptr;
    A.mode = 0;
    // exponentiation only (mont_mul/mont_sqr results are always canonical): 4N <= W^NP
    A.lazy = (c->bits + 2 <= 32u * c->np) ? 1 : 0;
}

void mpg::ctx_args(KArgs &A, const mont_ctx *c) { fill_ctx_args(A, c); }

// kernels for a Montgomery product or exponentiation on context c: MP_ALGO_KARATSUBA selects
// the truncated Karatsuba form (Sec. 5.1), which exists for the truncated reduction of the
// classes from 512 to 4096 bits; AUTO and SCHOOLBOOK the schoolbook shapes; null otherwise
static const ShapeOps *ops_for(const mont_ctx *c, mp_red red, mp_algo algo) {
    if (algo == MP_ALGO_KARATSUBA2) return nullptr;
    const SizeClass *cls = class_for(c->np);
    const bool tk_ok = red == MP_RED_TRUNCATED && cls && cls->tk.mont && (uint32_t)cls->tk.NP == c->np;
    if (algo == MP_ALGO_KARATSUBA) return tk_ok ? &cls->tk : nullptr;
    if (algo == MP_ALGO_AUTO && tk_ok && cls->mont_kara_from && c->bits >= cls->mont_kara_from) return &cls->tk;
    return shape_for_red(c->np, (int)red);
}

static int mont_common(uint32_t *out, const uint32_t *a, const uint32_t *b, const mont_ctx *c, mp_red red,
                       mp_algo algo, bool square, void *stream) {
    if (!out || !a || (!square && !b) || !c) return MP_ERR_ARG;
    if (red != MP_RED_TRUNCATED && red != MP_RED_FULL && red != MP_RED_CIOS) return MP_ERR_ARG;
    if (algo != MP_ALGO_AUTO && algo != MP_ALGO_SCHOOLBOOK && algo != MP_ALGO_KARATSUBA &&
        algo != MP_ALGO_KARATSUBA2)
        return MP_ERR_ARG;
    const ShapeOps *sh = ops_for(c, red, algo);
    if (!sh) return MP_ERR_UNIMPLEMENTED;
    if (c->layout == MP_LAYOUT_INTERLEAVED && (!aligned16(out) || !aligned16(a) || (!square && !aligned16(b))))
        return MP_ERR_ALIGN;
    KArgs A{};
    fill_ctx_args(A, c);
    A.out = out; A.a = a; A.b = square ? a : b; A.red = (int)red; A.square = square ? 1 : 0;
    return cuda_status(sh->mont(A, S(stream)));
}

extern "C" int mont_mul(uint32_t *out, const uint32_t *a, const uint32_t *b, const mont_ctx *c, mp_red red,
                        mp_algo algo, void *stream) {
    return mont_common(out, a, b, c, red, algo, false, stream);
}

extern "C" int mont_sqr(uint32_t *out, const uint32_t *a, const mont_ctx *c, mp_red red, mp_algo algo,
                        void *stream) {
    return mont_common(out, a, nullptr, c, red, algo, true, stream);
}

// ------------------------------------------------------------------ exponentiation

// window for window = 0: the tuned one for the size class, else 4 up to 1024 bits,
// 5 up to 3072, 6 above (Sec. 6.4 found 4 best at 1024 bits and 5 above)
// built-in window rule (measured on GB300, modexp/s: 1024 bits w = 4 1.662M, 3 1.585M, 5 1.631M;
// 2048 bits 5 314.0k, 4 313.0k; 3072 bits 5 96.8k, 4 95.8k; 4096 bits 5 42.1k, 6 39.7k)
static uint32_t tuned_window(uint32_t bits) {
    const SizeClass *c = class_for(words_for(bits));
    if (c && c->window) return c->window;
    return bits <= 1024 ? 4u : bits <= 4096 ? 5u : 6u;
}

uint32_t mpg::default_window(uint32_t bits) { return tuned_window(bits); }

const ShapeOps *mpg::shape_for_red_np(uint32_t np, int red) { return shape_for_red(np, red); }

extern "C" int mp_shape_candidates(uint32_t bits, int *G, int *M, int max) {
    if (bits == 0 || bits > MAX_BITS) return MP_ERR_SIZE;
    const SizeClass *c = class_for(words_for(bits));
    int k = 0;
    for (int i = 0; i < c->nshapes && k < max; ++i, ++k) {
        if (G) G[k] = c->shapes[i].G;
        if (M) M[k] = c->shapes[i].M;
    }
    return c->nshapes;
}

extern "C" int mp_tune_set(uint32_t bits, int G, int M, uint32_t window, uint32_t karatsuba_from_bits) {
    if (bits == 0 || bits > MAX_BITS) return MP_ERR_SIZE;
    if (window > 6) return MP_ERR_SIZE;
    SizeClass *c = class_for(words_for(bits));
    int pick = -1;
    for (int i = 0; i < c->nshapes; ++i)
        if (c->shapes[i].G == G && c->shapes[i].M == M) pick = i;
    if (G != 0 || M != 0) {
        if (pick < 0) return MP_ERR_ARG;
        c->chosen = pick;
    }
    c->window = window;
    c->kara_from = karatsuba_from_bits;
    return MP_OK;
}

extern "C" int mp_tune_get(uint32_t bits, int *G, int *M, uint32_t *window, uint32_t *karatsuba_from_bits) {
    if (bits == 0 || bits > MAX_BITS) return MP_ERR_SIZE;
    const SizeClass *c = class_for(words_for(bits));
    if (G) *G = c->shapes[c->chosen].G;
    if (M) *M = c->shapes[c->chosen].M;
    if (window) *window = tuned_window(bits);
    if (karatsuba_from_bits) *karatsuba_from_bits = c->kara_from ? c->kara_from : KARATSUBA_FROM_BITS;
    return MP_OK;
}

extern "C" int mp_tune_set_mont_karatsuba(uint32_t bits, uint32_t karatsuba_from_bits) {
    if (bits == 0 || bits > MAX_BITS) return MP_ERR_SIZE;
    class_for(words_for(bits))->mont_kara_from = karatsuba_from_bits;
    return MP_OK;
}

extern "C" int mp_tune_get_mont_karatsuba(uint32_t bits, uint32_t *karatsuba_from_bits) {
    if (bits == 0 || bits > MAX_BITS) return MP_ERR_SIZE;
    if (!karatsuba_from_bits) return MP_ERR_ARG;
    *karatsuba_from_bits = class_for(words_for(bits))->mont_kara_from;
    return MP_OK;
}

extern "C" int mp_tune_set_table(uint32_t bits, mp_table_placement placement) {
    if (bits == 0 || bits > MAX_BITS) return MP_ERR_SIZE;
    if (placement != MP_TABLE_GLOBAL && placement != MP_TABLE_SHARED) return MP_ERR_ARG;
    class_for(words_for(bits))->table_shared = placement == MP_TABLE_SHARED ? 1 : 0;
    return MP_OK;
}

extern "C" int mp_tune_get_table(uint32_t bits, mp_table_placement *placement) {
    if (bits == 0 || bits > MAX_BITS) return MP_ERR_SIZE;
    if (!placement) return MP_ERR_ARG;
    *placement = class_for(words_for(bits))->table_shared ? MP_TABLE_SHARED : MP_TABLE_GLOBAL;
    return MP_OK;
}

extern "C" int mp_table_residency(uint32_t bits, uint32_t window, int *instances_per_sm) {
    if (bits == 0 || bits > MAX_BITS) return MP_ERR_SIZE;
    if (!instances_per_sm || window == 0 || window > 6) return MP_ERR_ARG;
    const ShapeOps *sh = shape_for(words_for(bits));
    if (!sh || !sh->residency_tab) return MP_ERR_UNIMPLEMENTED;
    const int r = sh->residency_tab((int)window);
    if (r < 0) return MP_ERR_CUDA;
    *instances_per_sm = r;
    return MP_OK;
}

extern "C" int mp_shape_residency(uint32_t bits, int G, int M, mp_red red, mp_algo algo, int *instances_per_sm) {
    if (bits == 0 || bits > MAX_BITS) return MP_ERR_SIZE;
    if (!instances_per_sm || (red != MP_RED_TRUNCATED && red != MP_RED_FULL && red != MP_RED_CIOS)) return MP_ERR_ARG;
    const SizeClass *c = class_for(words_for(bits));
    const ShapeOps *sh = nullptr;
    if (algo == MP_ALGO_KARATSUBA) {
        if (red != MP_RED_TRUNCATED || !c->tk.modexp) return MP_ERR_UNIMPLEMENTED;
        sh = &c->tk;
    } else {
        for (int i = 0; i < c->nshapes; ++i)
            if (c->shapes[i].G == G && c->shapes[i].M == M) sh = &c->shapes[i];
        if (!sh) return MP_ERR_ARG;
    }
    if (!sh->residency) return MP_ERR_UNIMPLEMENTED;
    const int r = sh->residency((int)red);
    if (r < 0) return red == MP_RED_CIOS ? MP_ERR_UNIMPLEMENTED : MP_ERR_CUDA;
    *instances_per_sm = r;
    return MP_OK;
}

extern "C" size_t modexp_workspace_bytes(size_t batch, uint32_t bits, uint32_t window) {
    if (bits == 0 || bits > MAX_BITS) return 0;
    if (window == 0) window = tuned_window(bits);
    if (window > 6) return 0;
    const ShapeOps *sh = shape_for(words_for(bits));
    if (!sh) return 0;
    return ((size_t)1 << window) * (size_t)sh->NP * batch * 4;
}

extern "C" int modexp_consttime(uint32_t *y, const uint32_t *base, const uint32_t *exp, uint32_t exp_bits,
                                const mont_ctx *c, uint32_t window, mp_red red, mp_algo algo, void *workspace,
                                size_t workspace_bytes, void *stream) {
    if (!y || !base || !c || (exp_bits > 0 && !exp)) return MP_ERR_ARG;
    if (red != MP_RED_TRUNCATED && red != MP_RED_FULL && red != MP_RED_CIOS) return MP_ERR_ARG;
    if (algo != MP_ALGO_AUTO && algo != MP_ALGO_SCHOOLBOOK && algo != MP_ALGO_KARATSUBA &&
        algo != MP_ALGO_KARATSUBA2)
        return MP_ERR_ARG;
    const ShapeOps *sh = ops_for(c, red, algo);
    if (!sh) return MP_ERR_UNIMPLEMENTED;
    if (window == 0) window = tuned_window(c->bits);
    if (window > 6) return MP_ERR_SIZE;
    if (c->layout == MP_LAYOUT_INTERLEAVED && (!aligned16(y) || !aligned16(base) || (exp && !aligned16(exp))))
        return MP_ERR_ALIGN;
    const size_t need = modexp_workspace_bytes(c->batch, c->bits, window);
    cudaStream_t st = S(stream);
    void *ws = workspace;
    bool own = false;
    if (ws) {
        if (!aligned16(ws)) return MP_ERR_ALIGN;
        if (workspace_bytes < need) return MP_ERR_NOMEM;
    } else {
        if (cudaMallocAsync(&ws, need, st) != cudaSuccess) {
            cudaGetLastError();
            return MP_ERR_NOMEM;
        }
        own = true;
    }
    KArgs A{};
    fill_ctx_args(A, c);
    A.out = y; A.a = base; A.e = exp; A.table = reinterpret_cast<uint32_t *>(ws);
    A.ebits = (int)exp_bits; A.ne = exp_bits ? (int)((exp_bits + 31) / 32) : 1; A.window = (int)window;
    A.red = (int)red;
    A.tab_shared = class_for(c->np)->table_shared;
    int rc = cuda_status(sh->modexp(A, st));
    if (own) {
        if (cudaFreeAsync(ws, st) != cudaSuccess && rc == MP_OK) rc = MP_ERR_CUDA;
    }
    return rc;
}

// measurement helper of the constant-time test: modexp_consttime plus per-instance cycles
extern "C" int modexp_timing_probe(unsigned long long *cycles, uint32_t *y, const uint32_t *base, const uint32_t *exp,
                                   uint32_t exp_bits, const mont_ctx *c, uint32_t window, mp_red red, void *workspace,
                                   size_t workspace_bytes, void *stream) {
    if (!cycles || !y || !base || !c || !workspace || (exp_bits > 0 && !exp)) return MP_ERR_ARG;
    if (red != MP_RED_TRUNCATED && red != MP_RED_FULL && red != MP_RED_CIOS) return MP_ERR_ARG;
    const ShapeOps *sh = ops_for(c, red, MP_ALGO_AUTO);
    if (!sh) return MP_ERR_UNIMPLEMENTED;
    if (window == 0) window = tuned_window(c->bits);
    if (window > 6) return MP_ERR_SIZE;
    if (((uintptr_t)cycles & 7u) || !aligned16(workspace) ||
        (c->layout == MP_LAYOUT_INTERLEAVED && (!aligned16(y) || !aligned16(base) || (exp && !aligned16(exp)))))
        return MP_ERR_ALIGN;
    if (workspace_bytes < modexp_workspace_bytes(c->batch, c->bits, window)) return MP_ERR_NOMEM;
    KArgs A{};
    fill_ctx_args(A, c);
    A.out = y; A.a = base; A.e = exp; A.table = reinterpret_cast<uint32_t *>(workspace);
    A.ebits = (int)exp_bits; A.ne = exp_bits ? (int)((exp_bits + 31) / 32) : 1; A.window = (int)window;
    A.red = (int)red;
    A.cycles = cycles;
    return cuda_status(sh->modexp(A, S(stream)));
}

// ------------------------------------------------------------------ resident tables, fixed bases

extern "C" size_t modexp_table_bytes(const mont_ctx *c, uint32_t window) {
    if (!c || window == 0 || window > 6) return 0;
    return ((size_t)1 << window) * (size_t)c->np * c->batch * 4;
}

extern "C" int modexp_table_build(void *tables, size_t bytes, const uint32_t *base, const mont_ctx *c,
                                  uint32_t window, mp_red red, void *stream) {
    if (!tables || !base || !c) return MP_ERR_ARG;
    if (red != MP_RED_TRUNCATED && red != MP_RED_FULL && red != MP_RED_CIOS) return MP_ERR_ARG;
    if (window == 0 || window > 6) return MP_ERR_SIZE;
    if (!aligned16(tables) || (c->layout == MP_LAYOUT_INTERLEAVED && !aligned16(base))) return MP_ERR_ALIGN;
    if (bytes < modexp_table_bytes(c, window)) return MP_ERR_NOMEM;
    KArgs A{};
    fill_ctx_args(A, c);
    A.a = base; A.table = reinterpret_cast<uint32_t *>(tables); A.window = (int)window; A.red = (int)red;
    A.mode = 1;
    return cuda_status(shape_for_red(c->np, (int)red)->modexp(A, S(stream)));
}

extern "C" int modexp_fixed_base(uint32_t *y, const uint32_t *index, const uint32_t *exp, uint32_t exp_bits,
                                 size_t nreq, const mont_ctx *c, const void *tables, uint32_t window, mp_red red,
                                 void *stream) {
    if (!y || !index || !c || !tables || (exp_bits > 0 && !exp) || nreq == 0) return MP_ERR_ARG;
    if (red != MP_RED_TRUNCATED && red != MP_RED_FULL && red != MP_RED_CIOS) return MP_ERR_ARG;
    if (window == 0 || window > 6) return MP_ERR_SIZE;
    if (!aligned16(tables) || (c->layout == MP_LAYOUT_INTERLEAVED && (!aligned16(y) || (exp && !aligned16(exp)))))
        return MP_ERR_ALIGN;
    KArgs A{};
    fill_ctx_args(A, c);
    A.out = y; A.e = exp; A.index = index; A.batch = nreq;
    A.table = const_cast<uint32_t *>(reinterpret_cast<const uint32_t *>(tables));
    A.ebits = (int)exp_bits; A.ne = exp_bits ? (int)((exp_bits + 31) / 32) : 1; A.window = (int)window;
    A.red = (int)red;
    A.mode = 2;
    return cuda_status(shape_for_red(c->np, (int)red)->modexp(A, S(stream)));
}

// ------------------------------------------------------------------ exponentiation without allocation
//
// Window tables of modexp_consttime_noalloc live in this fixed device array
// instead of a caller workspace or a stream-ordered allocation. It is part of the
// library's device image, so every GPU that loads the library holds these bytes
// until the process exits. All calls share it and it keeps what the last call
// wrote; the exponentiation writes every table entry before reading it, so
// nothing needs clearing between calls. Two calls that overlap on the GPU (two
// streams, or two host threads) race on it.
static __device__ __align__(256) uint4 g_noalloc_tables[MPGPU_NOALLOC_SCRATCH_BYTES / 16];

static constexpr int NOALLOC_MAX_DEVICES = 64;

// The array's device address belongs to the context that loaded the library's device code
// into the device: after cudaDeviceReset the next primary context may place it elsewhere.
// The cache therefore keys each device's address by the id of the context current at the
// lookup (driver functions reached through the runtime, no link to the driver library).
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);
struct NoallocEntry {
    unsigned long long ctx_id;   // 0: empty
    uint32_t *ptr;
};
static NoallocEntry g_noalloc[NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mu;

// id of the context current on this thread
static int current_ctx_id(unsigned long long *id) {
    static CtxGetCurrentFn get_cur = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    CUcontext ctx = nullptr;
    if (!get_cur || !get_id || get_cur(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, id) != CUDA_SUCCESS) return MP_ERR_CUDA;
    return MP_OK;
}

// Device address of the array on the current device. In host code the array's name only
// stands for the device symbol, so the address comes from cudaGetSymbolAddress, taken with
// the device current, once per device and context.
static int noalloc_tables(uint32_t **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return MP_ERR_CUDA;
    if (cudaSetDevice(dev) != cudaSuccess) return MP_ERR_CUDA;   // makes the primary context current
    unsigned long long id = 0;
    if (current_ctx_id(&id) != MP_OK) return MP_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocEntry &e = g_noalloc[dev];
    if (e.ctx_id != id || !e.ptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_tables) != cudaSuccess || !p) {
            cudaGetLastError();
            return MP_ERR_CUDA;
        }
        e.ptr = reinterpret_cast<uint32_t *>(p);
        e.ctx_id = id;
    }
    *out = e.ptr;
    return MP_OK;
}

extern "C" size_t mp_noalloc_scratch_bytes(void) { return (size_t)MPGPU_NOALLOC_SCRATCH_BYTES; }

extern "C" int modexp_consttime_noalloc(uint32_t *y, const uint32_t *base, const uint32_t *exp, uint32_t exp_bits,
                                        const mont_ctx *c, uint32_t window, mp_red red, mp_algo algo,
                                        void *stream) {
    if (!y || !base || !c || (exp_bits > 0 && !exp)) return MP_ERR_ARG;
    if (red != MP_RED_TRUNCATED && red != MP_RED_FULL && red != MP_RED_CIOS) return MP_ERR_ARG;
    if (algo != MP_ALGO_AUTO && algo != MP_ALGO_SCHOOLBOOK && algo != MP_ALGO_KARATSUBA &&
        algo != MP_ALGO_KARATSUBA2)
        return MP_ERR_ARG;
    const ShapeOps *sh = ops_for(c, red, algo);
    if (!sh) return MP_ERR_UNIMPLEMENTED;
    if (window == 0) window = tuned_window(c->bits);
    if (window > 6) return MP_ERR_SIZE;
    if (c->layout == MP_LAYOUT_INTERLEAVED && (!aligned16(y) || !aligned16(base) || (exp && !aligned16(exp))))
        return MP_ERR_ALIGN;
    if (modexp_workspace_bytes(c->batch, c->bits, window) > (size_t)MPGPU_NOALLOC_SCRATCH_BYTES) return MP_ERR_SIZE;
    uint32_t *tables = nullptr;
    int rc = noalloc_tables(&tables);
    if (rc != MP_OK) return rc;
    KArgs A{};
    fill_ctx_args(A, c);
    A.out = y; A.a = base; A.e = exp; A.table = tables;
    A.ebits = (int)exp_bits; A.ne = exp_bits ? (int)((exp_bits + 31) / 32) : 1; A.window = (int)window;
    A.red = (int)red;
    return cuda_status(sh->modexp(A, S(stream)));
}

// ------------------------------------------------------------------ debug builds

#ifdef MPG_DEBUG_BOUNDS
// records one violation without making the access it describes (the checks' own test)
__global__ void k_dbg_selftest() {
    if (threadIdx.x == 0 && blockIdx.x == 0) dbg_ok(false, DBG_SELFTEST, 12345ull);
}
#endif

extern "C" int mp_debug_bounds(unsigned long long *first) {
#ifdef MPG_DEBUG_BOUNDS
    if (!first) return MP_ERR_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return MP_ERR_CUDA;
    init_classes();
    unsigned long long v = 0;
    auto take = [&](unsigned long long x) {
        if (!v) v = x;
    };
    for (auto &c : g_classes) {
        for (int i = 0; i < c.nshapes; ++i)
            if (c.shapes[i].dbg) take(c.shapes[i].dbg());
        if (c.tk.dbg) take(c.tk.dbg());
    }
    take(dbg_take_kara2());
    take(dbg_take());   // this unit's own kernels (conversion, context set-up)
    *first = v;
    return MP_OK;
#else
    (void)first;
    return MP_ERR_UNIMPLEMENTED;
#endif
}

extern "C" int mp_debug_bounds_selftest(void *stream) {
#ifdef MPG_DEBUG_BOUNDS
    k_dbg_selftest<<<1, 32, 0, S(stream)>>>();
    return cuda_status(cudaGetLastError());
#else
    (void)stream;
    return MP_ERR_UNIMPLEMENTED;
#endif
}
