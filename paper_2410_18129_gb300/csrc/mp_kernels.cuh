// Batched kernels built on the group arithmetic of mp_group.cuh, templated on the
// group shape (G threads x M words per instance). Each shape is instantiated in
// its own translation unit (mp_shape_*.cu) and exposed through a ShapeOps table.
#pragma once
#include <cuda_runtime.h>
#include <atomic>
#include <cstddef>
#include "mp_group.cuh"

namespace mpg {

enum { LAYOUT_IM = 0, LAYOUT_IL = 1 };

// word i of instance k in an array of `words` words per instance
MPG_DI size_t widx(int layout, size_t k, int i, int words, size_t batch) {
    return layout == LAYOUT_IM ? k * (size_t)words + (size_t)i
                               : (((size_t)(i >> 2) * batch + k) << 2) + (size_t)(i & 3);
}

// x[j] = word (w0 + j) of instance k, zero beyond `words` or for an invalid instance
template <int M>
MPG_DI void gload(uint32_t (&x)[M], const uint32_t *p, int layout, size_t k, bool valid, int w0,
                  int words, size_t batch) {
#ifdef MPG_DEBUG_BOUNDS
    if (valid && !dbg_ok(k < batch && w0 >= 0, DBG_LOAD, k)) valid = false;
#endif
    if constexpr (M % 4 == 0) {
        if (layout == LAYOUT_IL && (w0 & 3) == 0) {
#pragma unroll
            for (int c = 0; c < M / 4; ++c) {
                const int i = w0 + 4 * c;
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (valid && i < words) v = reinterpret_cast<const uint4 *>(p)[(size_t)(i >> 2) * batch + k];
                x[4 * c] = v.x;
                x[4 * c + 1] = (i + 1 < words) ? v.y : 0u;
                x[4 * c + 2] = (i + 2 < words) ? v.z : 0u;
                x[4 * c + 3] = (i + 3 < words) ? v.w : 0u;
            }
            return;
        }
    }
#pragma unroll
    for (int j = 0; j < M; ++j) {
        const int i = w0 + j;
        x[j] = (valid && i < words) ? p[widx(layout, k, i, words, batch)] : 0u;
    }
}

template <int M>
MPG_DI void gstore(uint32_t *p, const uint32_t (&x)[M], int layout, size_t k, bool valid, int w0, int words,
                   size_t batch) {
#ifdef MPG_DEBUG_BOUNDS
    if (valid && !dbg_ok(k < batch && w0 >= 0, DBG_STORE, k)) valid = false;
#endif
    if (!valid) return;
    if constexpr (M % 4 == 0) {
        if (layout == LAYOUT_IL && (w0 & 3) == 0) {
#pragma unroll
            for (int c = 0; c < M / 4; ++c) {
                const int i = w0 + 4 * c;
                if (i + 3 < words) {
                    reinterpret_cast<uint4 *>(p)[(size_t)(i >> 2) * batch + k] =
                        make_uint4(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
                } else {
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if (i + r < words) p[widx(layout, k, i + r, words, batch)] = x[4 * c + r];
                }
            }
            return;
        }
    }
#pragma unroll
    for (int j = 0; j < M; ++j) {
        const int i = w0 + j;
        if (i < words) p[widx(layout, k, i, words, batch)] = x[j];
    }
}

struct KArgs {
    uint32_t *out;
    const uint32_t *a;
    const uint32_t *b;
    const uint32_t *e;       // exponents (API layout, ne words)
    // context arrays: interleaved layout, NP words per instance
    const uint32_t *N;
    const uint32_t *NI;
    const uint32_t *R1;
    const uint32_t *R2;
    const uint32_t *K;
    uint32_t *table;         // window tables: [entry][NP/4][instances] uint4, one per request (mode 0)
                             // or per context instance (modes 1, 2)
    size_t batch;            // instances of the API arrays (requests)
    int n;                   // API words per value
    int layout;              // API layout
    int ebits, ne, window, red, square, correct;
    const uint32_t *index;   // routed requests: request k uses context instance index[k]
    size_t cbatch;           // instances of the context arrays and tables (== batch without index)
    int mode;                // exponentiation: 0 build the table and run, 1 build only, 2 run on a resident table
    int lazy;                // exponentiation: 4N <= W^NP, products skip the final subtraction (results < 2N)
    unsigned long long *cycles;   // measurement only: per request, SM clock cycles of its exponentiation
    int tab_shared;          // exponentiation, mode 0: the window tables in shared memory (table unused)
};

// instance of this thread within its block, and its thread index within the instance
template <class S>
MPG_DI int local_instance() {
    if constexpr (S::WMAP) return (int)(threadIdx.x & 31);   // lane = instance, warp = thread
    else return (int)(threadIdx.x / S::G);                   // G consecutive lanes per instance
}

template <class S>
MPG_DI Grp<S> make_group(uint32_t *smem) {
    Grp<S> g;
    g.sm = smem + local_instance<S>() * S::WORDS;
    g.pa = g.sm + S::OFF_P;
    if constexpr (S::WMAP) {
        g.t = (int)(threadIdx.x >> 5);
        g.gbase = 0;
    } else {
        g.t = threadIdx.x % S::G;
        g.gbase = (threadIdx.x & 31) & ~(S::G - 1);
    }
    return g;
}

// instances per block: TPB/G either way (with the warp mapping a block is G warps = 32 instances)
template <class S, int TPB>
MPG_DI size_t global_instance() {
    static_assert(!S::WMAP || TPB == 32 * S::G, "warp mapping: one block = G warps");
    return (size_t)blockIdx.x * (TPB / S::G) + local_instance<S>();
}

// load M words per thread of an API operand into shared memory
template <class S>
MPG_DI void load_api(const Grp<S> &g, uint32_t *dst, const uint32_t *src, const KArgs &A, size_t k, bool valid) {
    uint32_t x[S::M];
    gload<S::M>(x, src, A.layout, k, valid, g.t * S::M, A.n, A.batch);
    sts<S::M>(dst + g.t * S::M, x);
}

template <class S>
MPG_DI void load_ctx(const Grp<S> &g, uint32_t *dst, const uint32_t *src, const KArgs &A, size_t k, bool valid) {
    uint32_t x[S::M];
    gload<S::M>(x, src, LAYOUT_IL, k, valid, g.t * S::M, S::NP, A.cbatch);
    sts<S::M>(dst + g.t * S::M, x);
}

// Blocks per SM that the shared memory of a shape allows (228 KB per SM, 1 KB of it reserved per
// block), but never so many that a thread gets fewer than 64 registers. Montgomery kernels (MONT)
// of shapes with more than 16 words per thread keep 200: their exponentiation measured 29 % slower
// at 140 registers than at about 220, while their plain products run faster at the higher
// occupancy. The kernels declare it as their minimum blocks per SM, so the compiler may use every
// register that this occupancy leaves.
template <class S, int TPB, bool MONT = true>
constexpr int blocks_per_sm() {
    constexpr long smem = (long)(TPB / S::G) * S::WORDS * 4 + 1024;
    constexpr long by_smem = 233472L / smem;
    constexpr long min_regs = (MONT && S::M > 16) ? 200L : 64L;
    constexpr long by_regs = 65536L / (TPB * min_regs);
    constexpr long b = by_smem < by_regs ? by_smem : by_regs;
    return b < 1 ? 1 : (int)b;
}

// ------------------------------------------------------------------ mp_mul / mp_sqr

template <class S, int TPB>
__global__ void __launch_bounds__(TPB, (blocks_per_sm<S, TPB, false>())) k_mul(KArgs A) {
    extern __shared__ uint4 smem4[];
    Grp<S> g = make_group<S>(reinterpret_cast<uint32_t *>(smem4));
    const size_t k = global_instance<S, TPB>();
    const bool valid = k < A.batch;
    load_api<S>(g, g.X(), A.a, A, k, valid);
    if (!A.square) load_api<S>(g, g.Y(), A.b, A, k, valid);
    g.sync();
    if (A.square) phase_sqr<S>(g, g.X(), g.X(), g.T());   // squares in X, Y
    else phase_mul<S>(g, g.X(), g.Y(), g.T());
    // store 2n words
    uint32_t x[2 * S::M];
    lds<2 * S::M>(x, g.T() + 2 * g.t * S::M);
    gstore<2 * S::M>(A.out, x, A.layout, k, valid, 2 * g.t * S::M, 2 * A.n, A.batch);
}

// ------------------------------------------------------------------ mont_mul / mont_sqr

template <class S, int TPB, int RED>
__global__ void __launch_bounds__(TPB, (blocks_per_sm<S, TPB>())) k_mont(KArgs A) {
    extern __shared__ uint4 smem4[];
    Grp<S> g = make_group<S>(reinterpret_cast<uint32_t *>(smem4));
    const size_t k = global_instance<S, TPB>();
    const bool valid = k < A.batch;
    load_ctx<S>(g, g.N(), A.N, A, k, valid);
    load_ctx<S>(g, g.NI(), A.NI, A, k, valid);
    load_api<S>(g, g.X(), A.a, A, k, valid);
    if (!A.square) load_api<S>(g, g.Y(), A.b, A, k, valid);
    g.sync();
    mont_prepare<S, RED>(g);
    // one call site; a second product when the internal radix W^NP differs from the
    // API radix W^n: multiply by W^(2NP-n) mod N
    for (int r = 0; r <= (A.correct ? 1 : 0); ++r) {
        if (r) {
            load_ctx<S>(g, g.Y(), A.K, A, k, valid);
            g.sync();
        }
        mont_mul<S, RED>(g, r == 0 && A.square != 0, false);
    }
    uint32_t x[S::M];
    lds<S::M>(x, g.X() + g.t * S::M);
    gstore<S::M>(A.out, x, A.layout, k, valid, g.t * S::M, A.n, A.batch);
}

// ------------------------------------------------------------------ modexp

template <class S>
MPG_DI size_t tidx4(int e, int chunk, size_t k, size_t batch) {
    return ((size_t)e * (S::NP / 4) + (size_t)chunk) * batch + k;
}

// constant-time window value b: bits [pos, pos+w) of the exponent, zero at or above ebits
MPG_DI uint32_t window_bits(const KArgs &A, size_t k, bool valid, int pos, int w) {
    if (!valid) return 0u;
    const int wi = pos >> 5, sh = pos & 31;
    const uint32_t lo = (wi < A.ne) ? A.e[widx(A.layout, k, wi, A.ne, A.batch)] : 0u;
    const uint32_t hi = (wi + 1 < A.ne) ? A.e[widx(A.layout, k, wi + 1, A.ne, A.batch)] : 0u;
    uint32_t v = (uint32_t)((((uint64_t)hi << 32) | lo) >> sh) & ((1u << w) - 1u);
    const int keep = A.ebits - pos;   // public
    if (keep < w) v &= (1u << keep) - 1u;
    return v;
}

// One group's constant-time exponentiation (Alg. 7) of request k. Request k uses
// context instance kc = index[k] (requests routed to a resident pool of moduli) or k.
//   mode 0: build the window table of request k's base, then run the windows
//   mode 1: only build the table (a resident table for later fixed-base requests)
//   mode 2: run the windows on the resident table of instance kc
template <class S, int RED>
MPG_DI void modexp_group(const Grp<S> &g, const KArgs &A, size_t k) {
    constexpr int M = S::M;
    bool valid = k < A.batch;
    const size_t kc = (A.index && valid) ? (size_t)A.index[k] : k;   // routing: public
    valid = valid && kc < A.cbatch;
    const int w = A.window;
    const int E = 1 << w;
    // window table and base: per request when the job builds its tables (mode 0, also when
    // its requests are routed to context instances), per context instance for resident tables
    const size_t kt = A.mode == 0 ? k : kc;
    const size_t tb = A.mode == 0 ? A.batch : A.cbatch;
    uint4 *tab = reinterpret_cast<uint4 *>(A.table);

    auto put = [&](int e, const uint32_t *src) {   // this thread's M words -> table entry e
        uint32_t x[M];
        lds<M>(x, src + g.t * M);
#ifdef MPG_DEBUG_BOUNDS
        if (valid && !dbg_ok(e >= 0 && e < E && kt < tb, DBG_TABLE, (unsigned long long)e * tb + kt)) return;
#endif
        if (!valid) return;
        if constexpr (M % 4 == 0) {
#pragma unroll
            for (int c = 0; c < M / 4; ++c)
                tab[tidx4<S>(e, g.t * (M / 4) + c, kt, tb)] =
                    make_uint4(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
        } else {
#pragma unroll
            for (int j = 0; j < M; ++j) {
                const int i = g.t * M + j;
                A.table[tidx4<S>(e, i >> 2, kt, tb) * 4 + (i & 3)] = x[j];
            }
        }
    };
    auto fetch = [&](int e, uint32_t (&x)[M]) {     // table entry e -> this thread's M words
#ifdef MPG_DEBUG_BOUNDS
        if (valid && !dbg_ok(e >= 0 && e < E && kt < tb, DBG_TABLE, (unsigned long long)e * tb + kt)) {
            zero<M>(x);
            return;
        }
#endif
        if constexpr (M % 4 == 0) {
#pragma unroll
            for (int c = 0; c < M / 4; ++c) {
                uint4 v = make_uint4(0, 0, 0, 0);
                if (valid) v = tab[tidx4<S>(e, g.t * (M / 4) + c, kt, tb)];
                x[4 * c] = v.x; x[4 * c + 1] = v.y; x[4 * c + 2] = v.z; x[4 * c + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < M; ++j) {
                const int i = g.t * M + j;
                x[j] = valid ? A.table[tidx4<S>(e, i >> 2, kt, tb) * 4 + (i & 3)] : 0u;
            }
        }
    };

    load_ctx<S>(g, g.N(), A.N, A, kc, valid);
    load_ctx<S>(g, g.NI(), A.NI, A, kc, valid);
    // The products of the job, in order, run from ONE call site (one copy of the
    // Montgomery product in the instruction stream):
    //   build (modes 0, 1): G[1] = a * R^2, then G[e] = G[e-1] * G[1] for e = 2..E-1
    //   windows (modes 0, 2): per window w squarings, then the product with the scanned entry
    //   last: the product with 1 (leaves the Montgomery domain)
    // Which product comes next depends only on public sizes.
    const int nbuild = A.mode != 2 ? E - 1 : 0;
    const int windows = (A.ebits + w - 1) / w;
    const int nwin = A.mode != 1 ? windows * (w + 1) + 1 : 0;
    if (A.mode != 2) {
        load_api<S>(g, g.X(), A.a, A, kt, valid);
        load_ctx<S>(g, g.Y(), A.R2, A, kc, valid);
    } else {
        load_ctx<S>(g, g.X(), A.R1, A, kc, valid);     // Y_acc = 1 in Montgomery form
    }
    g.sync();
    mont_prepare<S, RED>(g);
    for (int op = 0; op < nbuild + nwin; ++op) {
        bool square = false;
        if (op >= nbuild) {
            const int r = op - nbuild;
            const int i = r / (w + 1), s = r - i * (w + 1);
            if (i == windows) {                         // the product with 1
                uint32_t x[M];
                zero<M>(x);
                if (g.t == 0) x[0] = 1u;
                sts<M>(g.Y() + g.t * M, x);
                g.sync();
            } else if (s < w) {
                square = true;
            } else {   // masked scan of the whole table: every entry is read, one is kept
                const uint32_t bsel = window_bits(A, k, valid, (windows - 1 - i) * w, w);
                uint32_t acc[M];
                zero<M>(acc);
                for (int e = 0; e < E; ++e) {
                    const uint32_t m = mask_if_equal((uint32_t)e, bsel);
                    uint32_t x[M];
                    fetch(e, x);
#pragma unroll
                    for (int j = 0; j < M; ++j) acc[j] |= x[j] & m;
                }
                sts<M>(g.Y() + g.t * M, acc);
                g.sync();
            }
        }
        mont_mul<S, RED>(g, square, A.lazy != 0);
        if (op < nbuild) {
            put(op + 1, g.X());
            if (op == 0) {                              // G[0] = R mod N
                load_ctx<S>(g, g.Y(), A.R1, A, kc, valid);
                put(0, g.Y());
            }
            if (op + 1 < nbuild) {                      // next: G[op+2] = G[op+1] * G[1]
                uint32_t x[M];                          // (the product leaves q in Y)
                fetch(1, x);
                sts<M>(g.Y() + g.t * M, x);
            } else if (A.mode == 0) {
                load_ctx<S>(g, g.X(), A.R1, A, kc, valid);   // Y_acc = 1 in Montgomery form
            }
            g.sync();
        }
    }
    if (A.mode == 1) return;
    if (A.lazy) cond_sub<S>(g, g.X(), 0u, g.N(), g.X());   // X <= N here: canonical result
    uint32_t x[M];
    lds<M>(x, g.X() + g.t * M);
    gstore<M>(A.out, x, A.layout, k, valid, g.t * M, A.n, A.batch);
}

template <class S, int TPB, int RED>
__global__ void __launch_bounds__(TPB, (blocks_per_sm<S, TPB>())) k_modexp(KArgs A) {
    extern __shared__ uint4 smem4[];
    Grp<S> g = make_group<S>(reinterpret_cast<uint32_t *>(smem4));
    const size_t k = global_instance<S, TPB>();
    const long long t0 = clock64();
    modexp_group<S, RED>(g, A, k);
    if (A.cycles && g.t == 0 && k < A.batch) A.cycles[k] = (unsigned long long)(clock64() - t0);
}

// ------------------------------------------------------------------ per-shape launch table

struct ShapeOps {
    int G, M, NP, tpb;
    size_t smem_bytes;
    cudaError_t (*mul)(const KArgs &, cudaStream_t);
    cudaError_t (*mont)(const KArgs &, cudaStream_t);
    cudaError_t (*modexp)(const KArgs &, cudaStream_t);
    cudaError_t (*kara)(const KArgs &, cudaStream_t);   // one-level Karatsuba product, or null
    int (*residency)(int red);   // instances per SM of the exponentiation kernel for reduction red (< 0: error)
    // instances per SM of the truncated exponentiation with its window tables in shared memory at
    // window w (0: the tables do not fit; < 0: error), or null when the shape has no such kernel
    int (*residency_tab)(int w);
    // debug builds: takes (reads and clears) the first bounds violation recorded by the kernels of
    // this shape's translation unit (0: none); null in release builds
    unsigned long long (*dbg)();
};

// resident instances per SM of a kernel with tpb threads, smem bytes of dynamic shared memory and
// per_block instances per block, on the current device
template <class F>
static int resident_instances(F kern, int tpb, size_t smem, int per_block) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, tpb, smem) != cudaSuccess) return -1;
    return blocks * per_block;
}

// Allow `smem` bytes of dynamic shared memory for kern on the current device, once per kernel
// and device (function attributes belong to a device's context, so a process that drives several
// GPUs sets each). done: one bit per device; two threads that race on a first call both set the
// attribute, which is harmless.
template <class F>
static cudaError_t smem_attr_once(std::atomic<unsigned long long> &done, F kern, size_t smem) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

// KIND tells the kernels of one shape apart, so that each gets its own attribute call
template <class S, int TPB, int KIND, class F>
static cudaError_t launch_k(F kern, const KArgs &A, cudaStream_t st) {
    constexpr int GPB = TPB / S::G;
    const size_t smem = (size_t)GPB * S::WORDS * 4;
    static std::atomic<unsigned long long> attr_done{0ull};
    const cudaError_t e = smem_attr_once(attr_done, kern, smem);
    if (e != cudaSuccess) return e;
    const size_t blocks = (A.batch + GPB - 1) / GPB;
    kern<<<(unsigned)blocks, TPB, smem, st>>>(A);
    return cudaGetLastError();
}

template <class S, int TPB>
struct ShapeImpl {
    static cudaError_t mul(const KArgs &A, cudaStream_t st) { return launch_k<S, TPB, 0>(k_mul<S, TPB>, A, st); }
    static cudaError_t mont(const KArgs &A, cudaStream_t st) {
        if constexpr (S::WMAP) {   // CIOS runs on the lane-mapped shapes only (the API picks one)
            if (A.red == 2) return cudaErrorNotSupported;
        } else {
            if (A.red == 2) return launch_k<S, TPB, 5>(k_mont<S, TPB, 2>, A, st);
        }
        return A.red ? launch_k<S, TPB, 3>(k_mont<S, TPB, 1>, A, st) : launch_k<S, TPB, 1>(k_mont<S, TPB, 0>, A, st);
    }
    static cudaError_t modexp(const KArgs &A, cudaStream_t st) {
        if constexpr (S::WMAP) {
            if (A.red == 2) return cudaErrorNotSupported;
        } else {
            if (A.red == 2) return launch_k<S, TPB, 6>(k_modexp<S, TPB, 2>, A, st);
        }
        return A.red ? launch_k<S, TPB, 4>(k_modexp<S, TPB, 1>, A, st) : launch_k<S, TPB, 2>(k_modexp<S, TPB, 0>, A, st);
    }
    static int residency(int red) {
        constexpr size_t smem = (size_t)(TPB / S::G) * S::WORDS * 4;
        constexpr int per = TPB / S::G;
        if constexpr (S::WMAP) {
            if (red == 2) return -1;
        } else {
            if (red == 2) return resident_instances(k_modexp<S, TPB, 2>, TPB, smem, per);
        }
        return red ? resident_instances(k_modexp<S, TPB, 1>, TPB, smem, per)
                   : resident_instances(k_modexp<S, TPB, 0>, TPB, smem, per);
    }
    static ShapeOps ops() {
        // the warp-mapped variant of a shape reports G < 0 (see mp_shape_candidates)
        return ShapeOps{S::WMAP ? -S::G : S::G, S::M, S::NP, TPB, (size_t)(TPB / S::G) * S::WORDS * 4, &mul, &mont,
                        &modexp, nullptr, &residency, nullptr, MPG_DBG_TAKE};
    }
};

}  // namespace mpg

#define MPG_DEFINE_SHAPE(G, M, TPB)                                              \
    namespace mpg {                                                              \
    ShapeOps shape_ops_##G##_##M() { return ShapeImpl<Shape<G, M>, TPB>::ops(); } \
    }

// the warp-mapped variant of shape (G, M): thread t of each instance is warp t of a block of G
// warps, lane = instance (32 instances per block)
#define MPG_DEFINE_SHAPE_W(G, M)                                                                          \
    namespace mpg {                                                                                       \
    ShapeOps shape_ops_##G##_##M##_w() { return ShapeImpl<Shape<G, M, true>, 32 * G>::ops(); }           \
    }

// a shape whose products can also run as one level of Karatsuba over the half shape (G, MH)
#define MPG_DEFINE_SHAPE_KARA(G, M, TPB, MH, TPBK)                                           \
    namespace mpg {                                                                          \
    ShapeOps shape_ops_##G##_##M() {                                                         \
        ShapeOps o = ShapeImpl<Shape<G, M>, TPB>::ops();                                     \
        o.kara = &launch_kara<Shape<G, M>, Shape<G, MH>, TPBK>;                              \
        return o;                                                                            \
    }                                                                                        \
    }
