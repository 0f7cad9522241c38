/*
 * mpgpu — batched multi-precision and Montgomery arithmetic on GB300 (sm_103a).
 *
 * C ABI of the library built from paper_2410_18129_gb300/csrc. Every entry point
 * works on a batch of independent instances ("8 values in parallel" in the
 * paper, Sec. 2; here any batch size). Values are little-endian arrays of
 * 32-bit words, n = ceil(bits/32) words per value; bits above `bits` must be 0.
 *
 * Conventions shared by every call
 *   - Data pointers are DEVICE pointers owned by the caller (e.g. torch tensors).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls are asynchronous on that stream and never synchronise it, except
 *     mont_ctx_init (documented there).
 *   - Return value: MP_OK (0) or a negative mp_status. Argument errors are
 *     detected on the host before any launch; launch failures map to MP_ERR_CUDA.
 *   - Layout (mp_layout) of an array of `batch` values of w words each:
 *       MP_LAYOUT_INSTANCE_MAJOR  word i of value k at  k*w + i            (GMP-like, Sec. 6.4)
 *       MP_LAYOUT_INTERLEAVED     word i of value k at  ((i/4)*batch + k)*4 + i%4
 *                                 (groups of four words of consecutive values side by side,
 *                                 the GPU analogue of the word slicing of Table 1); such an
 *                                 array holds ceil(w/4)*4*batch words.
 *   - Montgomery radix R = 2^(32n). Montgomery-domain values are x*R mod N.
 *     Every Montgomery output is canonical (< N): the library always performs the
 *     final conditional subtraction that Alg. 5 leaves optional, because R = 2^(32n)
 *     leaves no slack above a modulus whose top bit is set. Inside an exponentiation
 *     whose size is padded (4N <= 2^(32*NP), NP the padded word count of the size
 *     class) the products skip it and stay below 2N (the slack of Alg. 3/Alg. 5);
 *     the result is made canonical once at the end.
 *   - Preconditions of mont_* and modexp: inputs < N, N odd with its top bit (bits-1) set.
 *     Violations give unspecified (but memory-safe) results.
 */
#ifndef MPGPU_H
#define MPGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MP_OK = 0,
    MP_ERR_ARG = -1,            /* null pointer, zero batch, bad enum value */
    MP_ERR_SIZE = -2,           /* bits == 0 or above mp_max_bits(), window out of range */
    MP_ERR_EVEN_MODULUS = -3,   /* mont_ctx_init found an even modulus */
    MP_ERR_ALIGN = -4,          /* pointer not 16-byte aligned */
    MP_ERR_CUDA = -5,           /* a CUDA runtime call or kernel launch failed */
    MP_ERR_NOMEM = -6,          /* device allocation failed or workspace too small */
    MP_ERR_UNIMPLEMENTED = -7   /* combination the library does not provide */
} mp_status;

typedef enum { MP_LAYOUT_INSTANCE_MAJOR = 0, MP_LAYOUT_INTERLEAVED = 1 } mp_layout;
/* Products: schoolbook (Alg. 1/2), one level of Karatsuba (Sec. 3), two levels (mp_mul and
   mp_sqr of the 4096- and 4608-bit classes only; 9 quarter products instead of 16).
   For Montgomery products and exponentiation, MP_ALGO_KARATSUBA selects the truncated
   Karatsuba form (Sec. 5.1; see mont_mul). */
typedef enum { MP_ALGO_AUTO = 0, MP_ALGO_SCHOOLBOOK = 1, MP_ALGO_KARATSUBA = 2, MP_ALGO_KARATSUBA2 = 3 } mp_algo;
/* Reductions: truncated (Alg. 6), classical (Alg. 3/5), word-serial CIOS (Alg. 4). */
typedef enum { MP_RED_TRUNCATED = 0, MP_RED_FULL = 1, MP_RED_CIOS = 2 } mp_red;

/* Opaque per-batch Montgomery context: device copies of N, N', R mod N, R^2 mod N. */
typedef struct mont_ctx mont_ctx;

/* Human-readable text for a status code (static storage). */
const char *mp_strerror(int status);

/* Largest operand size in bits the library supports. */
uint32_t mp_max_bits(void);

/* Library version string (static storage). */
const char *mp_version(void);

/*
 * Layout conversion (the expand / contract step of Sec. 6.4, Table 8; here a
 * transpose, since the limb radix stays 2^32). dst and src hold `batch` values
 * of `words` words; dst and src must not overlap.
 */
int mp_convert(uint32_t *dst, mp_layout dst_layout, const uint32_t *src, mp_layout src_layout,
               size_t batch, uint32_t words, void *stream);

/*
 * Batch product C_k = A_k * B_k (Alg. 1 B_mul; Sec. 3 one-level Karatsuba).
 * a, b: n words per instance; c: 2n words per instance; all in `layout`.
 * algo: SCHOOLBOOK, KARATSUBA (one level, Sec. 3: three half-size products; sizes
 * above 512 bits, else MP_ERR_UNIMPLEMENTED), KARATSUBA2 (two levels, the 9 quarter
 * products of Sec. 3 applied twice; 4097..4608-bit and 3073..4096-bit sizes only, else
 * MP_ERR_UNIMPLEMENTED) or AUTO (schoolbook, the faster form on GB300 at every size, unless
 * mp_tune_set sets a Karatsuba switch-over for the class).
 * c must not overlap a or b.
 */
int mp_mul(uint32_t *c, const uint32_t *a, const uint32_t *b, size_t batch, uint32_t bits,
           mp_layout layout, mp_algo algo, void *stream);

/* Batch square C_k = A_k^2 (Alg. 2 B_square, Sec. 3). Same conventions as mp_mul. */
int mp_sqr(uint32_t *c, const uint32_t *a, size_t batch, uint32_t bits, mp_layout layout,
           mp_algo algo, void *stream);

/*
 * Build a Montgomery context for `batch` moduli N (n words each, `layout`):
 * N' = (-N)^{-1} mod R, R mod N and R^2 mod N (Sec. 4: the precomputed values of
 * Alg. 3 and the R^2 used to enter the Montgomery representation).
 * Allocates device memory (stream-ordered on `stream`; owned by the context until
 * mont_ctx_free) and synchronises `stream` to report moduli errors: if any N is even, returns
 * MP_ERR_EVEN_MODULUS, stores the smallest offending instance index in
 * *bad_index (when non-NULL) and creates no context. N is copied; the caller
 * may free it afterwards. Operands of later calls use the same `layout`.
 */
int mont_ctx_init(mont_ctx **ctx, const uint32_t *N, size_t batch, uint32_t bits,
                  mp_layout layout, size_t *bad_index, void *stream);

/* Free a context. Stream-ordered: the memory is returned after all work already queued on
   the stream given to mont_ctx_init, which must still exist; work that uses the context on
   other streams must be complete, or ordered before that point of the context's stream,
   when this is called. Nothing else waits. NULL is accepted. */
int mont_ctx_free(mont_ctx *ctx);

/* Context properties: batch, bits, layout. Any out pointer may be NULL. */
int mont_ctx_info(const mont_ctx *ctx, size_t *batch, uint32_t *bits, mp_layout *layout);

/*
 * Copy one context constant into a caller device buffer of n words per instance
 * in the context layout: which = 0 N', 1 R mod N, 2 R^2 mod N, 3 N.
 */
int mont_ctx_export(const mont_ctx *ctx, int which, uint32_t *dst, void *stream);

/*
 * Batch Montgomery product c_k = a_k * b_k * R^{-1} mod N_k (Alg. 3 with B_mul,
 * Alg. 5/6): red = MP_RED_TRUNCATED computes only the low half of q = T*N' mod R
 * and only the high half of q*N (Alg. 6, Thm. 1, Thm. 2); MP_RED_FULL forms the
 * whole T + q*N (Alg. 3, B_fma); MP_RED_CIOS interleaves the product and the
 * reduction word by word (Alg. 4: per word a_i, Y += a_i*B, q = (Y mod W)*n0',
 * Y = (Y + q*N)/W; needs only n0' = N' mod W). All give the same canonical result.
 * algo: AUTO or SCHOOLBOOK; or KARATSUBA with MP_RED_TRUNCATED for contexts of 257 to
 * 4096 bits (padded sizes 16 to 128 words): T by one Karatsuba level,
 * q from the low half of a Karatsuba product, and the high half of q*N in the truncated
 * Karatsuba form of Sec. 5.1 (D2 in full, column estimates of D0 and D1, the missing
 * carry recovered from word n-1 of -T). Other combinations return MP_ERR_UNIMPLEMENTED.
 * a, b, c: n words per instance in the context layout; c may alias a or b.
 */
int mont_mul(uint32_t *c, const uint32_t *a, const uint32_t *b, const mont_ctx *ctx, mp_red red,
             mp_algo algo, void *stream);

/* Batch Montgomery square c_k = a_k^2 * R^{-1} mod N_k (Alg. 2 then Alg. 5/6). */
int mont_sqr(uint32_t *c, const uint32_t *a, const mont_ctx *ctx, mp_red red, mp_algo algo,
             void *stream);

/*
 * Device workspace (bytes) that modexp_consttime needs for the window tables of
 * `batch` instances of `bits` bits at window width `window` (1..6).
 */
size_t modexp_workspace_bytes(size_t batch, uint32_t bits, uint32_t window);

/*
 * Constant-time fixed-window left-to-right exponentiation y_k = base_k^{e_k} mod N_k
 * (Alg. 7). exp holds ceil(exp_bits/32) words per instance (context layout);
 * exp_bits is public and fixes the work: ceil(exp_bits/window) windows, each of
 * `window` Montgomery squarings and one Montgomery product with a table entry
 * chosen by a masked scan of the whole table (no secret-dependent branch or
 * address). window = 0 picks the tuned width. base and y: n words per instance,
 * ordinary residues (converted to and from the Montgomery domain inside).
 * workspace: device buffer of at least modexp_workspace_bytes(...) bytes, 16-byte
 * aligned; workspace == NULL makes the call allocate and free it on `stream`
 * (stream-ordered allocation). y may alias base. red and algo as for mont_mul (every
 * product of the exponentiation uses them).
 */
int modexp_consttime(uint32_t *y, const uint32_t *base, const uint32_t *exp, uint32_t exp_bits,
                     const mont_ctx *ctx, uint32_t window, mp_red red, mp_algo algo,
                     void *workspace, size_t workspace_bytes, void *stream);

/*
 * Mixed-size batches (pattern (2) of the serving/batching use of Alg. 7): each job is
 * one context's batch of exponentiations, with its own operand size, exponent length
 * and window (0 = tuned), run with the kernel modexp_consttime would use for it (the
 * shape selected for its size class). Any size the library supports, at most 16 jobs
 * per call. The jobs are independent: the call forks them onto parallel streams of the
 * library, the costliest job first, and joins them back to `stream` with events, so the
 * GPU fills the last partial wave of one job with blocks of the next, and the call
 * (fork, launches, join) can be captured in a CUDA graph together with its copies.
 * Results equal those of modexp_consttime on each job.
 * red: MP_RED_TRUNCATED, MP_RED_FULL or MP_RED_CIOS, for every job of the call.
 * workspace: at least modexp_mixed_workspace_bytes(jobs, njobs) bytes, 256-byte
 * aligned (the window tables of the jobs that are not fixed-base).
 * The first call on a device creates that device's streams and events (outside any
 * stream capture); calls from several host threads are serialised around the fork.
 */
typedef struct {
    uint32_t *y;            /* results, n words per instance, context layout */
    const uint32_t *base;   /* bases < N (unused for fixed-base jobs) */
    const uint32_t *exp;    /* ceil(exp_bits/32) words per instance */
    uint32_t exp_bits;      /* public exponent length */
    uint32_t window;        /* 1..6, 0 = tuned (fixed-base jobs: the tables' window) */
    const mont_ctx *ctx;
    /* routed job when index != NULL: nreq requests, request i uses context instance index[i]
       (its modulus; a resident pool of moduli); y and exp then hold nreq instances.
       With tables != NULL the job is fixed-base: request i runs on the resident table of
       instance index[i] (see modexp_table_build) and base is unused. With tables == NULL
       request i brings its own base (base holds nreq instances) and its table is built in
       the workspace like an ordinary job's. */
    const uint32_t *index;
    const void *tables;
    size_t nreq;
} mp_modexp_job;
size_t modexp_mixed_workspace_bytes(const mp_modexp_job *jobs, int njobs);
int modexp_consttime_mixed(const mp_modexp_job *jobs, int njobs, mp_red red, void *workspace,
                           size_t workspace_bytes, void *stream);

/*
 * Resident window tables for fixed bases (serving: each modulus of a pool keeps its
 * base's table on the device, so a request costs only the window loop of Alg. 7).
 * modexp_table_bytes: device bytes of the tables of every instance of ctx at width
 * `window` (1..6). modexp_table_build: tables[k] = base_k^i * R mod N_k, i < 2^window,
 * for every instance k of ctx (base in the context layout).
 * modexp_fixed_base: y_i = base_{index[i]}^{e_i} mod N_{index[i]} for nreq requests;
 * index: nreq words (instance numbers < batch of ctx); y and exp: nreq instances in
 * the context layout; `window` must be the one the tables were built with. The same
 * constant-time window loop and masked scan as modexp_consttime; index values are
 * public routing data. Out-of-range indexes leave their outputs unwritten.
 */
size_t modexp_table_bytes(const mont_ctx *ctx, uint32_t window);
int modexp_table_build(void *tables, size_t bytes, const uint32_t *base, const mont_ctx *ctx,
                       uint32_t window, mp_red red, void *stream);
int modexp_fixed_base(uint32_t *y, const uint32_t *index, const uint32_t *exp, uint32_t exp_bits,
                      size_t nreq, const mont_ctx *ctx, const void *tables, uint32_t window, mp_red red,
                      void *stream);

/*
 * Tuning (process-wide; set it before issuing work, not concurrently with it).
 * Every operand size maps to a size class (its padded word count); a class has one
 * or more compiled group shapes: G threads cooperate on one instance, each holding
 * M words. mp_shape_candidates lists them (default first; returns how many); G < 0
 * names the same shape with thread t of every instance in warp t of its block (the lane
 * is the instance), which makes every branch on the thread index warp-uniform.
 * mp_tune_set selects the shape (G = M = 0 keeps it), the default window width of
 * modexp_consttime for window = 0 (0: built-in rule) and the size from which
 * MP_ALGO_AUTO products use Karatsuba (0: built-in rule) for the class of `bits`.
 * Contexts stay valid across changes (their layout depends on the class only).
 */
int mp_shape_candidates(uint32_t bits, int *G, int *M, int max);
int mp_tune_set(uint32_t bits, int G, int M, uint32_t window, uint32_t karatsuba_from_bits);
int mp_tune_get(uint32_t bits, int *G, int *M, uint32_t *window, uint32_t *karatsuba_from_bits);
/*
 * Montgomery products and exponentiations of the truncated reduction with MP_ALGO_AUTO use the
 * truncated Karatsuba form (Sec. 5.1, as MP_ALGO_KARATSUBA) from `karatsuba_from_bits` bits in
 * the class of `bits` (0: never, the built-in rule; sizes without the form keep schoolbook).
 */
int mp_tune_set_mont_karatsuba(uint32_t bits, uint32_t karatsuba_from_bits);
int mp_tune_get_mont_karatsuba(uint32_t bits, uint32_t *karatsuba_from_bits);
/*
 * Instances of the exponentiation kernel that fit on one SM at once (the occupancy of the
 * kernel that modexp_consttime runs for shape (G, M) of the class of `bits` with reduction
 * `red`; MP_ALGO_KARATSUBA: the truncated Karatsuba form's kernel, G and M ignored), on the
 * current device. A batch that is a multiple of this times the SM count runs in whole rounds.
 * MP_ERR_ARG for a shape the class does not have, MP_ERR_UNIMPLEMENTED for a combination
 * without a kernel.
 */
int mp_shape_residency(uint32_t bits, int G, int M, mp_red red, mp_algo algo, int *instances_per_sm);
/*
 * Window-table placement of modexp_consttime (Alg. 7's precomputed powers) for the class of
 * `bits`: MP_TABLE_GLOBAL (the default) keeps each instance's 2^w entries in the caller's
 * workspace and scans them from L2/HBM; MP_TABLE_SHARED keeps them in shared memory beside the
 * instance's record, for the truncated reduction on the role-swapped kernels, at windows whose
 * tables fit one block of 32 instances in an SM's shared memory (other calls keep the global
 * placement; the workspace argument stays required either way). A shared table costs occupancy:
 * 2^w x NP words per instance. mp_table_residency gives the instances per SM of that kernel at
 * window w on the current device (0: the tables do not fit), for the class's selected shape;
 * MP_ERR_UNIMPLEMENTED when that shape has no such kernel.
 */
typedef enum { MP_TABLE_GLOBAL = 0, MP_TABLE_SHARED = 1 } mp_table_placement;
int mp_tune_set_table(uint32_t bits, mp_table_placement placement);
int mp_tune_get_table(uint32_t bits, mp_table_placement *placement);
int mp_table_residency(uint32_t bits, uint32_t window, int *instances_per_sm);

/*
 * Debug builds only (the library compiled with -DMPG_DEBUG_BOUNDS, e.g. by
 * build.build(debug=True) into paper_2410_18129_gb300/_build_debug/): the kernels check
 * their shared-memory block accesses (inside the block's shared memory, 16-byte aligned
 * for vector accesses), the instance and word offsets of their global loads and stores,
 * and the window-table entries of the exponentiations. A failed check records its first
 * occurrence (kind in bits 56-63: 1 shared memory, 2 alignment, 3 load, 4 store, 5 table,
 * 6 self-test; the offending offset below) and skips the access; nothing traps.
 * mp_debug_bounds synchronises the device and returns the first recorded violation in
 * *first (0: none), clearing the record; mp_debug_bounds_selftest launches a kernel that
 * records one self-test violation without making any access. Release builds return
 * MP_ERR_UNIMPLEMENTED from both.
 */
int mp_debug_bounds(unsigned long long *first);
int mp_debug_bounds_selftest(void *stream);

/*
 * modexp_consttime without any device allocation. The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory on the
 * call path, e.g. a service that reserved its whole memory budget up front, code
 * that cannot afford the device-wide synchronisation and unpredictable latency of
 * cudaMalloc/cudaFree, or a host process whose device memory belongs to another
 * allocator. Same arguments and results as modexp_consttime minus the workspace:
 * the window tables go to one static device array of MPGPU_NOALLOC_SCRATCH_BYTES
 * bytes inside the library (every GPU that loads the library holds it until the
 * process exits). The call allocates nothing; the context still comes from
 * mont_ctx_init, done beforehand.
 *   - Limit: modexp_workspace_bytes(batch, bits, window) must not exceed
 *     MPGPU_NOALLOC_SCRATCH_BYTES (16 MiB: e.g. 2048 instances of 2048 bits at w=5,
 *     512 of 4096 bits at w=6; mp_noalloc_scratch_bytes() returns it); larger batches
 *     return MP_ERR_SIZE before any work.
 *   - The first call on a device looks up the array's device address (with that device
 *     current, then cached for the device's context; a new context, e.g. after
 *     cudaDeviceReset, looks it up again); make that first call before any stream
 *     capture.
 *   - All calls share the array, which keeps the last call's contents (each call
 *     writes every table entry before reading it). Calls that overlap on the GPU
 *     (concurrent streams or host threads) race on it: serialise them.
 */
#define MPGPU_NOALLOC_SCRATCH_BYTES (16u << 20)
/* Bytes of the static array of modexp_consttime_noalloc (MPGPU_NOALLOC_SCRATCH_BYTES of the
   library as built). */
size_t mp_noalloc_scratch_bytes(void);
int modexp_consttime_noalloc(uint32_t *y, const uint32_t *base, const uint32_t *exp, uint32_t exp_bits,
                             const mont_ctx *ctx, uint32_t window, mp_red red, mp_algo algo, void *stream);

/*
 * Measurement helper (no counterpart in the paper; it sets the roofline): runs one
 * block of 1024 threads per SM executing `iters` rounds of an integer instruction
 * mix and returns the issued rate per SM per clock (lanes x instructions / cycles,
 * from clock64) and the SM clock implied by the kernel's wall time.
 * mode 0: independent mad.lo.u32; 1: independent mad.hi.u32; 2: the library's 8x8
 * block product (mad.lo.cc/madc.hi.cc chains, counts its 128 multiply-adds);
 * 3: add.cc/addc.cc chains; 4: mad.wide.u32 chains fed by their own low word (counted as 2); 5: 8x8 block
 * product from mad.wide.u32 and 64-bit carry adds; 6: two independent 8x8 chain
 * products per iteration; 7: mode 2 on 256 threads per SM; 8: 10x10 block of 26-bit
 * digits summed into 64-bit columns by mad.wide.u32 (counted as 2 per product);
 * 9 / 10: 8x8 / 4x4 block products summed into one running split-column accumulator
 * (768 threads per SM); 11 / 12: the same with one array per block (block product plus
 * addition); 13 / 14: 4x4 blocks with one / two split accumulators on 256 threads per SM.
 * Synchronous; allocates a small scratch buffer.
 */
int mp_bench_imad(int mode, int iters, double *per_clk_per_sm, double *sm_mhz, void *stream);

/*
 * Measurement helper of the constant-time test (no counterpart in the paper; it checks
 * the constant-time claim of Alg. 7): modexp_consttime with the caller's workspace and
 * MP_ALGO_AUTO, writing also cycles[k] = SM clock cycles (clock64) from the start to the
 * end of instance k's exponentiation, for each of the ctx's instances (cycles: device,
 * batch 64-bit words, 8-byte aligned). Results in y as modexp_consttime's.
 */
int modexp_timing_probe(unsigned long long *cycles, uint32_t *y, const uint32_t *base, const uint32_t *exp,
                        uint32_t exp_bits, const mont_ctx *ctx, uint32_t window, mp_red red,
                        void *workspace, size_t workspace_bytes, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MPGPU_H */
