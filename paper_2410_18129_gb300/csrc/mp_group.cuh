// Group-cooperative multi-precision arithmetic: one instance per group of G
// threads of a warp, each thread holding M consecutive words of every operand.
//
// Products are computed as sums of B x B "block products" (B = M for full
// products, B = M/2 for the truncated halves). Output columns are cut into
// slots of B words; every thread owns two slots chosen so that all threads do
// the same number of block products (balanced even for the triangular low and
// high halves) and accumulates each slot in registers. When a slot is complete
// its low B words go straight to the phase's output array and its spill (the
// words above, B+1 of them) to a small shared area. A carry-resolution pass then
// adds each predecessor's spill, passes a small overflow word to the successor
// through a shuffle, and resolves the remaining one-bit carries for the whole
// group at once with warp ballots (carry-lookahead).
//
// Montgomery product (Alg. 5 / Alg. 6 in 32-bit words, R = 2^(32*NP)):
//   1. T = X*Y            (Alg. 1) or T = X^2 (Alg. 2)
//   2. q = T_lo * N' mod R          (low half only)
//   3a. truncated: C = T_hi + floor(q*N/R) + c_add           (Alg. 6, Thm. 1, Thm. 2)
//   3b. classical: C = (T + q*N) / R                         (Alg. 3 with B_fma)
//   4. C >= N ? C - N : C  (constant-time select)
// No branch or address depends on operand values; branches on the thread
// index inside the group (which slot a thread owns) are public.
#pragma once
#include "mp_limb.cuh"

// loops over block products stay loops: one copy of the block product per phase
#define MPG_BLOCK_LOOP _Pragma("unroll 1")

// block-wide barrier of the warp mapping (a checking build may supply its own)
#ifndef MPG_BLOCK_BARRIER
#define MPG_BLOCK_BARRIER() __syncthreads()
#endif

namespace mpg {

// W_ = false: the G threads of an instance are G consecutive lanes of a warp (a warp holds
// 32/G instances). W_ = true: thread t of an instance is warp t of its block and the lane is
// the instance (a block of G warps holds 32 instances), so every branch on the thread index
// is uniform across a warp; the threads of an instance then talk through shared memory and
// block barriers instead of shuffles and ballots.
template <int G_, int M_, bool W_ = false>
struct Shape {
    static constexpr int G = G_;           // threads per instance
    static constexpr int M = M_;           // words per thread
    static constexpr bool WMAP = W_;       // thread index = warp index (see above)
    static constexpr int NP = G * M;       // words per operand (padded size)
    static constexpr int H = M / 2;        // half-block width of the truncated products
    static constexpr int A1 = 2 * M + 2;   // slot accumulator words, full blocks
    static constexpr int A2 = 2 * H + 2;   // slot accumulator words, half blocks
    static_assert(G >= 2 && G <= 16 && (G & (G - 1)) == 0, "G must be 2, 4, 8 or 16");
    static_assert(M >= 2, "M must be >= 2");
    static constexpr bool MONT_OK = (M >= 4 && M % 2 == 0);   // half blocks of >= 2 words
    // per-instance shared memory map (32-bit words)
    static constexpr int OFF_X = 0;               // operand / result; X and Y together hold the block squares
    static constexpr int OFF_Y = NP;              // operand, then q
    static constexpr int OFF_N = 2 * NP;          // modulus
    static constexpr int OFF_NI = 3 * NP;         // N' = (-N)^-1 mod R
    static constexpr int OFF_T = 4 * NP;          // T (2*NP words)
    static constexpr int OFF_P = 6 * NP;          // slot spills: 2G slots of M words, then 2G top words
    static constexpr int OFF_XB = OFF_P + 2 * G * (M + 1);   // W_: one byte per thread (predicate exchange)
    static constexpr int OFF_XW = OFF_XB + (W_ ? (G + 3) / 4 : 0);   // W_: one broadcast word
    static constexpr int WORDS_RAW = OFF_XW + (W_ ? 1 : 0);
    // Instance stride (words), a multiple of 4 (16-byte aligned instances).
    // Lane mapping: a half-warp's 8-byte accesses (spill words, carries) touch 16/G instances
    // at the same offsets; a stride of 2G (mod 32) words spreads them evenly over the 32 banks
    // (G = 16: one instance per half-warp; 16 (mod 32) separates the two of a warp).
    // Warp mapping: 32 lanes read the same offset of 32 instances; a stride of 4 (mod 8)
    // words puts 8 lanes' 16-byte loads on distinct banks.
    static constexpr int BANK_RES = G < 16 ? 2 * G : 16;
    static constexpr int WORDS_A = (WORDS_RAW + 3) & ~3;
    static constexpr int WORDS = W_ ? ((WORDS_RAW + 3) / 8) * 8 + 4
                                    : WORDS_A + ((BANK_RES - WORDS_A % 32) % 32 + 32) % 32;
};

// Per-thread view of its group.
template <class S>
struct Grp {
    uint32_t *sm;   // this instance's shared words
    uint32_t *pa;   // slot spill area (2G slots of B words, then 2G top words; B = block width)
    int t;          // thread index in the group
    int gbase;      // warp lane of thread 0 of the group (lane mapping)
    MPG_DI uint32_t *X() const { return sm + S::OFF_X; }
    MPG_DI uint32_t *Y() const { return sm + S::OFF_Y; }
    MPG_DI uint32_t *Q() const { return sm + S::OFF_Y; }   // q reuses Y once T is formed
    MPG_DI uint32_t *N() const { return sm + S::OFF_N; }
    MPG_DI uint32_t *NI() const { return sm + S::OFF_NI; }
    MPG_DI uint32_t *T() const { return sm + S::OFF_T; }
    MPG_DI uint32_t *P() const { return pa; }
    // all threads of the group reach this point (and see each other's shared-memory writes)
    MPG_DI void sync() const {
        if constexpr (S::WMAP) MPG_BLOCK_BARRIER();
        else __syncwarp();
    }
    // m[k] bit u = p[k] of thread u of the group (collective: every thread calls it)
    template <int K>
    MPG_DI void bits(const bool (&p)[K], uint32_t (&m)[K]) const {
        static_assert(K <= 8, "at most 8 predicates");
        if constexpr (!S::WMAP) {
#pragma unroll
            for (int k = 0; k < K; ++k) m[k] = (__ballot_sync(0xffffffffu, p[k]) >> gbase) & ((1u << S::G) - 1u);
        } else {
            uint32_t b = 0u;
#pragma unroll
            for (int k = 0; k < K; ++k) b |= (p[k] ? 1u : 0u) << k;
            reinterpret_cast<uint8_t *>(sm + S::OFF_XB)[t] = (uint8_t)b;
            MPG_BLOCK_BARRIER();
            constexpr int NW = (S::G + 3) / 4;
            uint32_t w[NW];
#pragma unroll
            for (int i = 0; i < NW; ++i) w[i] = sm[S::OFF_XB + i];
#pragma unroll
            for (int k = 0; k < K; ++k) m[k] = 0u;
#pragma unroll
            for (int u = 0; u < S::G; ++u) {
                const uint32_t byte = w[u >> 2] >> (8 * (u & 3));
#pragma unroll
                for (int k = 0; k < K; ++k) m[k] |= ((byte >> k) & 1u) << u;
            }
            MPG_BLOCK_BARRIER();   // the exchange byte may be written again
        }
    }
    // the group's mask of one predicate (lane mapping only: a single ballot)
    MPG_DI uint32_t gbits(bool pred) const {
        static_assert(!S::WMAP, "use bits<K>() with the warp mapping");
        return (__ballot_sync(0xffffffffu, pred) >> gbase) & ((1u << S::G) - 1u);
    }
    // thread src's value v, for every thread of the group (collective)
    MPG_DI uint32_t bcast(uint32_t v, int src) const {
        if constexpr (!S::WMAP) {
            return __shfl_sync(0xffffffffu, v, gbase + src);
        } else {
            if (t == src) sm[S::OFF_XW] = v;
            MPG_BLOCK_BARRIER();
            const uint32_t r = sm[S::OFF_XW];
            MPG_BLOCK_BARRIER();
            return r;
        }
    }
};

MPG_DI void gsync() { __syncwarp(); }

// ------------------------------------------------------------------ shared-memory blocks

template <int K>
MPG_DI void lds(uint32_t (&x)[K], const uint32_t *p) {
#ifdef MPG_DEBUG_BOUNDS
    if (!smem_ok(p, 4 * K, K % 4 == 0)) {
#pragma unroll
        for (int k = 0; k < K; ++k) x[k] = 0u;
        return;
    }
#endif
    if constexpr (K % 4 == 0) {
#pragma unroll
        for (int k = 0; k < K / 4; ++k) {
            uint4 v = reinterpret_cast<const uint4 *>(p)[k];
            x[4 * k] = v.x; x[4 * k + 1] = v.y; x[4 * k + 2] = v.z; x[4 * k + 3] = v.w;
        }
    } else if constexpr (K % 2 == 0) {
#pragma unroll
        for (int k = 0; k < K / 2; ++k) {
            uint2 v = reinterpret_cast<const uint2 *>(p)[k];
            x[2 * k] = v.x; x[2 * k + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) x[k] = p[k];
    }
}

template <int K>
MPG_DI void sts(uint32_t *p, const uint32_t (&x)[K]) {
#ifdef MPG_DEBUG_BOUNDS
    if (!smem_ok(p, 4 * K, K % 4 == 0)) return;
#endif
    if constexpr (K % 4 == 0) {
#pragma unroll
        for (int k = 0; k < K / 4; ++k)
            reinterpret_cast<uint4 *>(p)[k] = make_uint4(x[4 * k], x[4 * k + 1], x[4 * k + 2], x[4 * k + 3]);
    } else if constexpr (K % 2 == 0) {
#pragma unroll
        for (int k = 0; k < K / 2; ++k) reinterpret_cast<uint2 *>(p)[k] = make_uint2(x[2 * k], x[2 * k + 1]);
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) p[k] = x[k];
    }
}

template <int K>
MPG_DI void zero(uint32_t (&x)[K]) {
#pragma unroll
    for (int k = 0; k < K; ++k) x[k] = 0u;
}

// a += X_u * Y_v for B-word blocks at p and q
template <int B>
MPG_DI void mac_block(Acc3<B> &a, const uint32_t *xp, const uint32_t *yp) {
    uint32_t x[B], y[B];
    lds<B>(x, xp);
    lds<B>(y, yp);
    acc3_mac<B>(a, x, y);
}

// mac_block with the product dropped when !live (the Y operand masked to zero), so that
// threads with fewer block products run the same instructions
template <int B>
MPG_DI void mac_block_live(Acc3<B> &a, const uint32_t *xp, const uint32_t *yp, bool live) {
    uint32_t x[B], y[B];
    lds<B>(x, xp);
    lds<B>(y, yp);
    const uint32_t m = live ? 0xffffffffu : 0u;
#pragma unroll
    for (int j = 0; j < B; ++j) y[j] &= m;
    acc3_mac<B>(a, x, y);
}

// a += X_{u(j)} * Y_{v(j)} for j = 0 .. cnt-1 (B-word blocks; uv(j, u, v) gives the pair), with
// the operands of step j+1 loaded from shared memory while step j multiplies (two register
// buffers, the loop unrolled by two so they alternate without moves). at(j) runs after step j.
template <int B, class UV, class AT>
MPG_DI void mac_loop_pipelined(Acc3<B> &V, const uint32_t *X, const uint32_t *Y, int cnt,
                               const UV &uv, const AT &at) {
    uint32_t xa[B], ya[B], xb[B], yb[B];
    int u, v;
    uv(0, u, v);
    lds<B>(xa, X + u * B);
    lds<B>(ya, Y + v * B);
    int j = 0;
    MPG_BLOCK_LOOP
    for (; j + 1 < cnt; j += 2) {
        uv(j + 1, u, v);
        lds<B>(xb, X + u * B);
        lds<B>(yb, Y + v * B);
        acc3_mac<B>(V, xa, ya);
        at(j);
        uv(j + 2 < cnt ? j + 2 : j + 1, u, v);   // the last pair reloads in-range operands
        lds<B>(xa, X + u * B);
        lds<B>(ya, Y + v * B);
        acc3_mac<B>(V, xb, yb);
        at(j + 1);
    }
    if (j < cnt) {
        acc3_mac<B>(V, xa, ya);
        at(j);
    }
}

// a += X_{u(j)} * Y_{v(j)} for j = 0 .. cnt-1: groups of U block products per iteration of a
// rolled loop, then the remaining cnt % U blocks straight-line. With a single block product
// per loop iteration the compiler splits the multiply-add pairs of the chains into separate
// lo and hi instructions (measured: 654 instead of 273 multiply-pipe instructions for 272
// partial products); with two full or four half blocks per iteration they stay paired.
// xm maps the word offset u*B of X's block u to its place in X (identity by default).
struct IdMap {
    MPG_DI int operator()(int i) const { return i; }
};

template <int B, int U, class UV, class XM = IdMap>
MPG_DI void mac_run(Acc3<B> &a, const uint32_t *X, const uint32_t *Y, int cnt, const UV &uv, const XM &xm = XM{}) {
    int j = 0;
    MPG_BLOCK_LOOP
    for (; j + U <= cnt; j += U) {
#pragma unroll
        for (int r = 0; r < U; ++r) {
            int u, v;
            uv(j + r, u, v);
            mac_block<B>(a, X + xm(u * B), Y + v * B);
        }
    }
#pragma unroll
    for (int r = 0; r + 1 < U; ++r) {
        if (j + r < cnt) {
            int u, v;
            uv(j + r, u, v);
            mac_block<B>(a, X + xm(u * B), Y + v * B);
        }
    }
}

// blocks per iteration of mac_run: two full blocks, four half blocks of up to 4 words
template <int B>
constexpr int run_group() { return B > 4 ? 2 : 4; }

// The double-buffered loop pays for 4-word half blocks (measured); with wider half blocks
// the extra registers cost more than the hidden load latency.
template <class S>
constexpr bool PIPELINE_HALF_BLOCKS = (S::H <= 4);

// ------------------------------------------------------------------ carry resolution

enum SlotPattern { PAT_SEQ = 0, PAT_ZIGZAG = 1, PAT_ONE = 2 };

template <int G, int PAT>
MPG_DI int slot_of(int t, int k) {
    if constexpr (PAT == PAT_SEQ) return k ? G + t : t;
    else if constexpr (PAT == PAT_ZIGZAG) return k ? 2 * G - 1 - t : t;
    else return t;
}

// group ballot bits (bit t = lane t of the group) -> bits indexed by slot number
template <int G, int PAT>
MPG_DI uint64_t slot_mask(uint32_t bitsA, uint32_t bitsB) {
    if constexpr (PAT == PAT_SEQ) return (uint64_t)bitsA | ((uint64_t)bitsB << G);
    else if constexpr (PAT == PAT_ZIGZAG) return (uint64_t)bitsA | ((uint64_t)(__brev(bitsB) >> (32 - 2 * G)));
    else return (uint64_t)bitsA;
}

struct NoXform {
    static constexpr bool active = false;
    template <int A>
    MPG_DI void operator()(int, uint32_t (&)[A]) const {}
};

// Spill area of slot s for B-word blocks: words B .. 2B-1 of the slot sum at P + s*B, word 2B
// at P + 2G*B + s. A slot sum stays below W^(2B+1) (at most 2(2G+1) block products of B x B
// words, or a doubled and offset square sum), so its word 2B+1 is zero and B+1 spill words hold
// the rest of it.
struct Spill {
    uint32_t *m;   // B words
    uint32_t *t;   // 1 word
};
template <class S, int B>
MPG_DI Spill spill_of(const Grp<S> &g, int s) {
    return Spill{g.P() + s * B, g.P() + 2 * S::G * B + s};
}

// store a slot sum: low B words to out_lo, the rest to the slot's spill area
template <int B>
MPG_DI void store_slot(const uint32_t (&V)[2 * B + 2], uint32_t *out_lo, Spill sp) {
    uint32_t lo[B], hi[B];
#pragma unroll
    for (int j = 0; j < B; ++j) { lo[j] = V[j]; hi[j] = V[B + j]; }
    sts<B>(out_lo, lo);
    sts<B>(sp.m, hi);
    *sp.t = V[2 * B];
}

// store a slot's running sum without clearing it. A thread accumulates its two slots in ONE
// register sum: it parks the sum when the first slot is complete and recovers the second slot
// at the end as the final sum minus the parked one (unpark_sub), so the loop body never clears
// registers.
template <int B>
MPG_DI void park(const Acc3<B> &a, uint32_t *out_lo, Spill sp) {
    uint32_t V[2 * B + 2];
    acc3_value<B>(V, a);
    store_slot<B>(V, out_lo, sp);
}

// complete slot s: store it and clear the accumulator
template <int B>
MPG_DI void flush(Acc3<B> &a, uint32_t *out_lo, Spill sp) {
    park<B>(a, out_lo, sp);
    acc3_zero<B>(a);
}

// the second slot of a parked sum: V = a - the sum parked at out_lo / spill, stored as slot s2
template <int B>
MPG_DI void unpark_store(const Acc3<B> &a, const uint32_t *out_lo, Spill sp, uint32_t *out2, Spill sp2);

// V -= the sum parked at out_lo / spill (exact: V holds the parked sum plus more)
template <int B>
MPG_DI void unpark_sub(uint32_t (&V)[2 * B + 2], const uint32_t *out_lo, Spill sp) {
    uint32_t lo[B], hi[B];
    lds<B>(lo, out_lo);
    lds<B>(hi, sp.m);
    const uint32_t top = *sp.t;
    sub_cc(V[0], lo[0]);
#pragma unroll
    for (int j = 1; j < B; ++j) subc_cc(V[j], lo[j]);
#pragma unroll
    for (int j = 0; j < B; ++j) subc_cc(V[B + j], hi[j]);
    subc_cc(V[2 * B], top);
    subc_cc(V[2 * B + 1], 0u);
}

template <int B>
MPG_DI void unpark_store(const Acc3<B> &a, const uint32_t *out_lo, Spill sp, uint32_t *out2, Spill sp2) {
    uint32_t V[2 * B + 2];
    acc3_value<B>(V, a);
    unpark_sub<B>(V, out_lo, sp);
    store_slot<B>(V, out2, sp2);
}

// overflow words of the predecessor slot, passed between lanes with shuffles
template <int G, int PAT>
MPG_DI void pred_overflow(int t, int gbase, const uint32_t (&ovA)[2], const uint32_t (&ovB)[2],
                          uint32_t (&inA)[2], uint32_t (&inB)[2]) {
#pragma unroll
    for (int w = 0; w < 2; ++w) {
        const uint32_t up = __shfl_sync(0xffffffffu, ovA[w], gbase + (t > 0 ? t - 1 : 0));
        inA[w] = t > 0 ? up : 0u;                                   // slot t <- slot t-1
        if constexpr (PAT == PAT_SEQ) {
            const uint32_t upB = __shfl_sync(0xffffffffu, ovB[w], gbase + (t > 0 ? t - 1 : 0));
            const uint32_t wrap = __shfl_sync(0xffffffffu, ovA[w], gbase + G - 1);
            inB[w] = t > 0 ? upB : wrap;                            // slot G+t <- G+t-1
        } else {
            const uint32_t dn = __shfl_sync(0xffffffffu, ovB[w], gbase + (t < G - 1 ? t + 1 : G - 1));
            inB[w] = t < G - 1 ? dn : ovA[w];                       // slot 2G-1-t <- 2G-2-t
        }
    }
}

// Turn completed slots (low B words already at OUT[s*B..], spill words at
// spill_of(s)) into words OUT[s*B..s*B+B). in0: B+2 words added below slot 0 (a
// carry coming from outside). xf may rewrite a slot sum first (add an addend,
// double it ...). Returns the low word of everything above the last slot (its own
// spill and overflow plus the resolved carry).
template <class S, int B, int PAT, class XF>
MPG_DI uint32_t resolve(const Grp<S> &g, const uint32_t (&in0)[B + 2], const XF &xf, uint32_t *OUT) {
    static_assert(PAT == PAT_SEQ || PAT == PAT_ZIGZAG, "two slots per thread");
    constexpr int G = S::G;
    constexpr int SP = B + 2;
    constexpr int NSLOT = 2 * G;
    uint32_t lo[2][B];
    uint32_t top = 0u;   // words at and above the last slot (owner lane only)

    // 1. optional per-slot rewrite; keep the low B words
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int s = slot_of<G, PAT>(g.t, k);
        const Spill sp = spill_of<S, B>(g, s);
        uint32_t V[2 * B + 2];
        {
            uint32_t l[B], h[B];
            lds<B>(l, OUT + s * B);
            lds<B>(h, sp.m);
#pragma unroll
            for (int j = 0; j < B; ++j) { V[j] = l[j]; V[B + j] = h[j]; }
            V[2 * B] = *sp.t;
            V[2 * B + 1] = 0u;
        }
        if constexpr (XF::active) {   // the rewritten sum stays below W^(2B+1) (see spill_of)
            xf(s, V);
            uint32_t h[B];
#pragma unroll
            for (int j = 0; j < B; ++j) h[j] = V[B + j];
            sts<B>(sp.m, h);
            *sp.t = V[2 * B];
        }
#pragma unroll
        for (int j = 0; j < B; ++j) lo[k][j] = V[j];
        if (s == NSLOT - 1) top = V[B];
    }
    if constexpr (XF::active) g.sync();
    // 2. add the predecessor's spill
    uint32_t ov[2][2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int s = slot_of<G, PAT>(g.t, k);
        uint32_t x[SP];
        if (s == 0) {
#pragma unroll
            for (int j = 0; j < SP; ++j) x[j] = in0[j];
        } else {
            const Spill pp = spill_of<S, B>(g, s - 1);
            uint32_t h[B];
            lds<B>(h, pp.m);
#pragma unroll
            for (int j = 0; j < B; ++j) x[j] = h[j];
            x[B] = *pp.t;
            x[B + 1] = 0u;
        }
        add_cc(x[0], lo[k][0]);
#pragma unroll
        for (int j = 1; j < B; ++j) addc_cc(x[j], lo[k][j]);
        addc_cc(x[B], 0u);
        addc(x[B + 1], 0u);
#pragma unroll
        for (int j = 0; j < B; ++j) lo[k][j] = x[j];
        ov[k][0] = x[B];
        ov[k][1] = x[B + 1];
        if (s == NSLOT - 1) top += x[B];
    }
    // 3. add the predecessor's overflow: leaves a 0/1 carry per slot
    uint32_t oin[2][2];
    if constexpr (!S::WMAP) {
        pred_overflow<G, PAT>(g.t, g.gbase, ov[0], ov[1], oin[0], oin[1]);
    } else {   // through the spill words, which every thread has read by now
        g.sync();
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            uint32_t *m = spill_of<S, B>(g, slot_of<G, PAT>(g.t, k)).m;
            m[0] = ov[k][0];
            m[1] = ov[k][1];
        }
        g.sync();
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int s = slot_of<G, PAT>(g.t, k);
            const uint32_t *m = spill_of<S, B>(g, s > 0 ? s - 1 : 0).m;
            oin[k][0] = s ? m[0] : 0u;
            oin[k][1] = s ? m[1] : 0u;
        }
    }
    uint32_t cgen[2], cprop[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        add_cc(lo[k][0], oin[k][0]);
        addc_cc(lo[k][1], oin[k][1]);
#pragma unroll
        for (int j = 2; j < B; ++j) addc_cc(lo[k][j], 0u);
        cgen[k] = addc_get();
        uint32_t all = lo[k][0];
#pragma unroll
        for (int j = 1; j < B; ++j) all &= lo[k][j];
        cprop[k] = (all == 0xffffffffu) ? 1u : 0u;
    }
    // 4. carry-lookahead over the slots: carry into slot s = bit s of ((P + 2G) ^ P)
    const bool pr[4] = {cgen[0] != 0u, cprop[0] != 0u, cgen[1] != 0u, cprop[1] != 0u};
    uint32_t mk[4];
    g.template bits<4>(pr, mk);
    const uint64_t Gm = slot_mask<G, PAT>(mk[0], mk[2]);
    const uint64_t Pmask = slot_mask<G, PAT>(mk[1], mk[3]);
    const uint64_t cin = (Pmask + (Gm << 1)) ^ Pmask;
    g.sync();   // every thread has read the spills it needs before OUT and P change again
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int s = slot_of<G, PAT>(g.t, k);
        add_word<B>(lo[k], (uint32_t)(cin >> s) & 1u);
        sts<B>(OUT + s * B, lo[k]);
    }
    // the carry out of the last slot; callers use it only where the value above it is 0 or 1
    constexpr int owner = (PAT == PAT_ZIGZAG) ? 0 : G - 1;
    top = g.bcast(top, owner);
    g.sync();
    return top + ((uint32_t)(cin >> NSLOT) & 1u);
}

// ------------------------------------------------------------------ products

// Slot sums of T = X * Y (2*NP words), stored unresolved (low words at T, spills in P).
// Full blocks: thread t owns slots t and G+t and computes X_j * Y_{(t-j) mod G} for
// j = 0..G-1 (G block products for every thread).
template <class S>
MPG_DI void mul_slots(const Grp<S> &g, const uint32_t *X, const uint32_t *Y, uint32_t *T) {
    constexpr int G = S::G, M = S::M;
    Acc3<M> V;
    acc3_zero<M>(V);
    const int t = g.t;
    if constexpr (S::WMAP) {   // t is uniform across the warp: one loop per slot
        MPG_BLOCK_LOOP
        for (int j = 0; j <= t; ++j) mac_block<M>(V, X + j * M, Y + (t - j) * M);
        flush<M>(V, T + t * M, spill_of<S, M>(g, t));
        MPG_BLOCK_LOOP
        for (int j = t + 1; j < G; ++j) mac_block<M>(V, X + j * M, Y + (t - j + G) * M);
        park<M>(V, T + (G + t) * M, spill_of<S, M>(g, G + t));
    } else {
        MPG_BLOCK_LOOP
        for (int j = 0; j < G; ++j) {
            const int v = (t - j) & (G - 1);
            mac_block<M>(V, X + j * M, Y + v * M);
            if (j == t) park<M>(V, T + t * M, spill_of<S, M>(g, t));
        }
        unpark_store<M>(V, T + t * M, spill_of<S, M>(g, t), T + (G + t) * M, spill_of<S, M>(g, G + t));
    }
}

// T = X * Y (2*NP words)
template <class S>
MPG_DI void phase_mul(const Grp<S> &g, const uint32_t *X, const uint32_t *Y, uint32_t *T) {
    constexpr int M = S::M;
    mul_slots<S>(g, X, Y, T);
    g.sync();
    uint32_t in0[M + 2];
    zero<M + 2>(in0);
    resolve<S, M, PAT_SEQ>(g, in0, NoXform{}, T);
}

// slot sums of squaring: V = 2 * (cross products) + (squares of the blocks)
template <class S>
struct SqrXform {
    static constexpr bool active = true;
    const uint32_t *D;
    template <int A>
    MPG_DI void operator()(int s, uint32_t (&V)[A]) const {
        constexpr int M = S::M;
#pragma unroll
        for (int k = A - 1; k > 0; --k) V[k] = __funnelshift_l(V[k - 1], V[k], 1);
        V[0] <<= 1;
        uint32_t d[M];
        lds<M>(d, D + s * M);
        add_cc(V[0], d[0]);
#pragma unroll
        for (int j = 1; j < M; ++j) addc_cc(V[j], d[j]);
#pragma unroll
        for (int j = M; j < A - 1; ++j) addc_cc(V[j], 0u);
        addc(V[A - 1], 0u);
    }
};

// Slot sums of the cross products of X^2 (Alg. 2 structure): X_u X_v, u < v, not yet
// doubled. Thread t owns slots t and G+t (pairs u < v with u + v = t and G + t).
template <class S>
MPG_DI void sqr_slots(const Grp<S> &g, const uint32_t *X, uint32_t *T) {
    constexpr int G = S::G, M = S::M;
    const int nA = (g.t + 1) >> 1;              // pairs u < v with u + v = t
    const int nB = ((G - g.t + 1) >> 1) - 1;    // pairs with u + v = G + t
    constexpr int K = G / 2;                    // max of nA + nB over the group
    Acc3<M> V;
    acc3_zero<M>(V);
    if constexpr (S::WMAP) {   // t is uniform across the warp: exact pair counts, no dummy blocks
        MPG_BLOCK_LOOP
        for (int j = 0; j < nA; ++j) mac_block<M>(V, X + j * M, X + (g.t - j) * M);
        flush<M>(V, T + g.t * M, spill_of<S, M>(g, g.t));
        MPG_BLOCK_LOOP
        for (int j = 0; j < nB; ++j) {
            const int u = g.t + 1 + j;
            mac_block<M>(V, X + u * M, X + (G + g.t - u) * M);
        }
        park<M>(V, T + (G + g.t) * M, spill_of<S, M>(g, G + g.t));
    } else {
        MPG_BLOCK_LOOP
        for (int j = 0; j < K; ++j) {
            if (j == nA) park<M>(V, T + g.t * M, spill_of<S, M>(g, g.t));
            int u, v;
            if (j < nA) { u = j; v = g.t - j; }
            else { u = g.t + 1 + (j - nA); v = G + g.t - u; }
            const bool live = j < nA + nB;
            mac_block_live<M>(V, X + (live ? u : 0) * M, X + (live ? v : 0) * M, live);
        }
        if (nA == K) park<M>(V, T + g.t * M, spill_of<S, M>(g, g.t));
        unpark_store<M>(V, T + g.t * M, spill_of<S, M>(g, g.t), T + (G + g.t) * M, spill_of<S, M>(g, G + g.t));
    }
}

// T = X^2: twice the cross products plus the squares of the G blocks. The block squares
// (one per thread) are formed after the cross products and parked side by side in D
// (2*NP words; D may overlap X); the resolve doubles each slot sum and adds them.
template <class S>
MPG_DI void phase_sqr(const Grp<S> &g, const uint32_t *X, uint32_t *D, uint32_t *T) {
    constexpr int M = S::M;
    sqr_slots<S>(g, X, T);
    uint32_t x[M], P[2 * M];
    lds<M>(x, X + g.t * M);
    g.sync();                                   // all reads of X are done
    block_sqr<M>(P, x);
    sts<2 * M>(D + 2 * g.t * M, P);
    g.sync();
    uint32_t in0[M + 2];
    zero<M + 2>(in0);
    resolve<S, M, PAT_SEQ>(g, in0, SqrXform<S>{D}, T);
}

// Slot sums of Q = (X * Y) mod W^NP with half blocks (H words, 2G of them). Thread t owns
// slots t and 2G-1-t: t+1 and 2G-t block products, 2G+1 for every thread.
template <class S>
MPG_DI void mullo_slots(const Grp<S> &g, const uint32_t *X, const uint32_t *Y, uint32_t *Q) {
    static_assert(S::MONT_OK, "Montgomery needs an even M >= 4");
    constexpr int G = S::G, H = S::H;
    Acc3<H> V;
    acc3_zero<H>(V);
    const int t = g.t;
    if constexpr (S::WMAP) {   // t is uniform across the warp: one loop per slot
        const auto none = [](int) {};
        mac_loop_pipelined<H>(V, X, Y, t + 1, [&](int j, int &u, int &v) { u = j; v = t - j; }, none);
        flush<H>(V, Q + t * H, spill_of<S, H>(g, t));
        mac_loop_pipelined<H>(V, X, Y, 2 * G - t, [&](int k, int &u, int &v) { u = k; v = 2 * G - t - 1 - k; },
                              none);
        park<H>(V, Q + (2 * G - 1 - t) * H, spill_of<S, H>(g, 2 * G - 1 - t));
    } else {
        const auto uv = [&](int j, int &u, int &v) {
            if (j <= t) { u = j; v = t - j; }
            else { u = j - t - 1; v = 2 * G - j; }
        };
        const auto at = [&](int j) { if (j == t) park<H>(V, Q + t * H, spill_of<S, H>(g, t)); };
        if constexpr (PIPELINE_HALF_BLOCKS<S>) {
            mac_loop_pipelined<H>(V, X, Y, 2 * G + 1, uv, at);
        } else {
            MPG_BLOCK_LOOP
            for (int j = 0; j <= 2 * G; ++j) {
                int u, v;
                uv(j, u, v);
                mac_block<H>(V, X + u * H, Y + v * H);
                at(j);
            }
        }
        unpark_store<H>(V, Q + t * H, spill_of<S, H>(g, t), Q + (2 * G - 1 - t) * H,
                        spill_of<S, H>(g, 2 * G - 1 - t));
    }
}

// Q = (X * Y) mod W^NP
template <class S>
MPG_DI void phase_mullo(const Grp<S> &g, const uint32_t *X, const uint32_t *Y, uint32_t *Q) {
    constexpr int H = S::H;
    mullo_slots<S>(g, X, Y, Q);
    g.sync();
    uint32_t in0[H + 2];
    zero<H + 2>(in0);
    resolve<S, H, PAT_ZIGZAG>(g, in0, NoXform{}, Q);
}

template <int B>
struct AddendXform {
    static constexpr bool active = true;
    const uint32_t *Add;   // B words per slot
    template <int A>
    MPG_DI void operator()(int s, uint32_t (&V)[A]) const {
        uint32_t d[B];
        lds<B>(d, Add + s * B);
        add_cc(V[0], d[0]);
#pragma unroll
        for (int j = 1; j < B; ++j) addc_cc(V[j], d[j]);
#pragma unroll
        for (int j = B; j < A - 1; ++j) addc_cc(V[j], 0u);
        addc(V[A - 1], 0u);
    }
};

// Z += the part of one H x H block product X_u*Y_v (u + v = 2G-1, so its local
// column c sits at global column NP-H+c) that Thm. 2 needs: lo halves of the pairs
// with i+j >= H-1 at word i+j-(H-1), hi halves of the pairs with i+j >= H-2 at word
// i+j-(H-2). Word 0 of Z is global column NP-1.
template <int H>
MPG_DI void tri_mac(uint32_t (&Z)[H + 3], const uint32_t *xp, const uint32_t *yp) {
    uint32_t x[H], y[H];
    lds<H>(x, xp);
    lds<H>(y, yp);
#pragma unroll
    for (int i = 0; i < H; ++i) {
        const int jl = (H - 1 - i > 0) ? H - 1 - i : 0;
#pragma unroll
        for (int j = jl; j < H; ++j) {
            if (j == jl) mad_lo_cc(Z[i + j - H + 1], x[i], y[j]);
            else madc_lo_cc(Z[i + j - H + 1], x[i], y[j]);
        }
#pragma unroll
        for (int p = i + 1; p < H + 3; ++p) addc_cc(Z[p], 0u);
        const int jh = (H - 2 - i > 0) ? H - 2 - i : 0;
#pragma unroll
        for (int j = jh; j < H; ++j) {
            if (j == jh) mad_hi_cc(Z[i + j - H + 2], x[i], y[j]);
            else madc_hi_cc(Z[i + j - H + 2], x[i], y[j]);
        }
#pragma unroll
        for (int p = i + 2; p < H + 3; ++p) addc_cc(Z[p], 0u);
    }
}

// Truncated high half (Alg. 6 lines 2-4 with Thm. 1 and Thm. 2), computing
//   C = floor(T / R) + floor(q*N / R) + c_add            (NP words + carry out)
// from only the partial products of q*N of weight >= NP-1 (lo halves) and
// >= NP-2 (hi halves):
//   * block products with u + v >= 2G (all their columns are >= NP) go to the
//     H-word output slots h = u+v-2G (slot h covers words NP + h*H ...);
//   * the blocks on the diagonal u + v = 2G-1 contribute their upper triangle
//     (tri_mac) and the blocks on u + v = 2G-2 their corner hi half (column NP-2)
//     to a small accumulator Z whose word 0 is column NP-1 (the sum S of Eq. qn);
//   * the carry into column NP-1 from below is unknown, but word NP-1 of q*N is
//     known: it is L = ((-T) mod R)[NP-1] (Thm. 1: T + qN = 0 mod R). Hence the
//     carry out of column NP-1 is floor(Z / W) plus one exactly when L < Z[0].
//
// mulhi_slots forms the parts that do not depend on T: the output slots (parked, not yet
// resolved) and this thread's share Z of the boundary sum (warp mapping: also parked in T's
// low half, dead once q is formed); mulhi_sums adds the shares over the group (lane mapping:
// every thread holds the sum; warp mapping: thread 0 does).
template <class S>
MPG_DI void mulhi_slots(const Grp<S> &g, const uint32_t *Qs, const uint32_t *Ns, uint32_t *C, uint32_t (&Z)[S::H + 3]) {
    constexpr int G = S::G, H = S::H, NP = S::NP;
    // column NP-1 and the hi halves that reach it: thread t takes diagonal blocks u = 2t, 2t+1
    zero<H + 3>(Z);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int u = 2 * g.t + j;
        tri_mac<H>(Z, Qs + u * H, Ns + (2 * G - 1 - u) * H);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {   // corners of the blocks u + v = 2G-2 (2G-1 of them)
        const int u = 2 * g.t + j;
        const bool live = u <= 2 * G - 2;
        const uint32_t xq = Qs[u * H + H - 1];
        const uint32_t yn = live ? Ns[(2 * G - 2 - u) * H + H - 1] : 0u;
        add_word<H + 3>(Z, __umulhi(xq, yn));
    }
    if constexpr (S::WMAP) {   // park Z in T's low half, dead since q was formed (T[NP-1] kept)
        static_assert(G * (H + 3) <= NP - 1, "Z exchange must stay below word NP-1 of T");
        uint32_t *zs = g.T() + g.t * (H + 3);
#pragma unroll
        for (int k = 0; k < H + 3; ++k) zs[k] = Z[k];
    }
    // output slots: A = t (absolute 2G+t), B = 2G-1-t (absolute 4G-1-t)
    Acc3<H> V;
    acc3_zero<H>(V);
    const int t = g.t;
    const int nA = 2 * G - 1 - t;
    if constexpr (S::WMAP) {   // t is uniform across the warp: one loop per slot
        const auto none = [](int) {};
        mac_loop_pipelined<H>(V, Qs, Ns, nA, [&](int j, int &u, int &v) { u = t + 1 + j; v = 2 * G - 1 - j; },
                              none);
        flush<H>(V, C + t * H, spill_of<S, H>(g, t));
        if (t > 0)   // slot B of thread t has t products (none for thread 0)
            mac_loop_pipelined<H>(V, Qs, Ns, t, [&](int k, int &u, int &v) { u = 2 * G - t + k; v = 2 * G - 1 - k; },
                                  none);
        park<H>(V, C + (2 * G - 1 - t) * H, spill_of<S, H>(g, 2 * G - 1 - t));
    } else {
        const auto uv = [&](int j, int &u, int &v) {
            if (j < nA) { u = t + 1 + j; v = 2 * G + t - u; }
            else { u = j + 1; v = 4 * G - 2 - t - j; }
        };
        const auto at = [&](int j) { if (j == nA - 1) park<H>(V, C + t * H, spill_of<S, H>(g, t)); };
        if constexpr (PIPELINE_HALF_BLOCKS<S>) {
            mac_loop_pipelined<H>(V, Qs, Ns, 2 * G - 1, uv, at);
        } else {
            MPG_BLOCK_LOOP
            for (int j = 0; j < 2 * G - 1; ++j) {
                int u, v;
                uv(j, u, v);
                mac_block<H>(V, Qs + u * H, Ns + v * H);
                at(j);
            }
        }
        unpark_store<H>(V, C + t * H, spill_of<S, H>(g, t), C + (2 * G - 1 - t) * H,
                        spill_of<S, H>(g, 2 * G - 1 - t));
    }
}

template <class S>
MPG_DI void mulhi_sums(const Grp<S> &g, const uint32_t *Qs, const uint32_t *Ns, uint32_t *C, uint32_t (&Z)[S::H + 3]) {
    constexpr int G = S::G, H = S::H;
    const int t = g.t;
    mulhi_slots<S>(g, Qs, Ns, C, Z);
    if constexpr (S::WMAP) {
        // thread 0 (owner of slot 0, the only one that needs the sum) adds the parked Z's
        g.sync();
        if (t == 0) {
#pragma unroll 1
            for (int u = 1; u < G; ++u) {
                uint32_t o[H + 3];
#pragma unroll
                for (int k = 0; k < H + 3; ++k) o[k] = g.T()[u * (H + 3) + k];
                add_n<H + 3>(Z, o);
            }
        }
    } else {   // sum Z over the group (butterfly; every lane gets the total)
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) {
            uint32_t o[H + 3];
#pragma unroll
            for (int k = 0; k < H + 3; ++k) o[k] = __shfl_xor_sync(0xffffffffu, Z[k], off);
            add_n<H + 3>(Z, o);
        }
    }
}

// C = floor(T/R) + floor(q*N/R) + c_add from the stored slots of the high half and the group
// sum Z (word 0 at column NP-1); returns the carry out of C
// (xf: the transform that adds T's high words to the slot sums, unless the slots already
// hold them)
template <class S, class XF>
MPG_DI uint32_t mulhi_resolve(const Grp<S> &g, const uint32_t (&Z)[S::H + 3], const uint32_t *T, uint32_t c_add,
                              uint32_t low_zero, uint32_t *C, const XF &xf) {
    constexpr int H = S::H, NP = S::NP;
    // L = ((-T) mod R)[NP-1] = ~T[NP-1] + [T[0 .. NP-1) == 0]  (mod W)
    const uint32_t L = ~T[NP - 1] + low_zero;
    const uint32_t extra = (uint32_t)(((uint64_t)L - (uint64_t)Z[0]) >> 63);   // [L < Z[0]]
    uint32_t in0[H + 2];
#pragma unroll
    for (int j = 0; j < H + 2; ++j) in0[j] = Z[1 + j];
    add_word<H + 2>(in0, extra + c_add);
    return resolve<S, H, PAT_ZIGZAG>(g, in0, xf, C);
}

template <class S>
MPG_DI uint32_t phase_mulhi(const Grp<S> &g, const uint32_t *Qs, const uint32_t *Ns, const uint32_t *T,
                            uint32_t c_add, uint32_t low_zero, uint32_t *C) {
    constexpr int H = S::H;
    uint32_t Z[H + 3];
    mulhi_sums<S>(g, Qs, Ns, C, Z);
    g.sync();
    return mulhi_resolve<S>(g, Z, T, c_add, low_zero, C, AddendXform<H>{T + S::NP});
}

// Column estimate of floor(X*Y / W^(NP-1)) from the same partial products (the truncated
// half product of the Karatsuba form, Sec. 5.1): words NP .. 2NP-1 go to C, word NP-1 is
// returned. Nothing below column NP-1 is known here, so no carry is recovered: the
// estimate is at most 2*NP below the exact value. Lane mapping only.
template <class S>
MPG_DI uint32_t phase_mulhi_est(const Grp<S> &g, const uint32_t *Xs, const uint32_t *Ys, uint32_t *C) {
    static_assert(!S::WMAP, "estimate: lane mapping only");
    constexpr int H = S::H;
    uint32_t Z[H + 3];
    mulhi_sums<S>(g, Xs, Ys, C, Z);
    uint32_t in0[H + 2];
#pragma unroll
    for (int j = 0; j < H + 2; ++j) in0[j] = Z[1 + j];
    g.sync();
    resolve<S, H, PAT_ZIGZAG>(g, in0, NoXform{}, C);
    return Z[0];
}

// Slot sums of the classical reduction T + q*N over all 2*NP words (B_fma): thread t's
// slots t and G+t, T's words of each slot added before it is stored over them.
template <class S>
MPG_DI void fma_slots(const Grp<S> &g, const uint32_t *Qs, const uint32_t *Ns, uint32_t *T) {
    constexpr int G = S::G, M = S::M, A = S::A1;
    Acc3<M> acc;
    acc3_zero<M>(acc);
    const AddendXform<M> addT{T};
    MPG_BLOCK_LOOP
    for (int j = 0; j < G; ++j) {
        const int v = (g.t - j) & (G - 1);
        mac_block<M>(acc, Qs + j * M, Ns + v * M);
        if (j == g.t) {   // add T's words of this slot, then store over them
            uint32_t V[A];
            acc3_value<M>(V, acc);
            addT(g.t, V);
            store_slot<M>(V, T + g.t * M, spill_of<S, M>(g, g.t));
            acc3_zero<M>(acc);
        }
    }
    {
        uint32_t V[A];
        acc3_value<M>(V, acc);
        addT(G + g.t, V);
        store_slot<M>(V, T + (G + g.t) * M, spill_of<S, M>(g, G + g.t));
    }
}

// Classical reduction: T + q*N, result in T. Returns the carry out of the top word
// (C = T[NP..2NP) + carry * R).
template <class S>
MPG_DI uint32_t phase_fma(const Grp<S> &g, const uint32_t *Qs, const uint32_t *Ns, uint32_t *T) {
    constexpr int M = S::M;
    fma_slots<S>(g, Qs, Ns, T);
    g.sync();
    uint32_t in0[M + 2];
    zero<M + 2>(in0);
    return resolve<S, M, PAT_SEQ>(g, in0, NoXform{}, T);
}

// OUT = (carry*R + C >= N) ? C - N : C, constant time. Borrows are resolved across
// the group with the same lookahead (a slot equal to N's propagates a borrow).
template <class S>
MPG_DI void cond_sub(const Grp<S> &g, const uint32_t *C, uint32_t carry, const uint32_t *Ns, uint32_t *OUT) {
    constexpr int G = S::G, M = S::M;
    uint32_t c[M], nn[M], d[M];
    lds<M>(c, C + g.t * M);
    lds<M>(nn, Ns + g.t * M);
    uint32_t eq = 0u;
#pragma unroll
    for (int j = 0; j < M; ++j) { d[j] = c[j]; eq |= c[j] ^ nn[j]; }
    const uint32_t bgen = sub_n<M>(d, nn);
    const bool pr[2] = {bgen != 0u, eq == 0u};
    uint32_t mk[2];
    g.template bits<2>(pr, mk);
    const uint32_t gb = mk[0], pb = mk[1];
    const uint64_t Pm = pb, Gm = gb;
    const uint64_t bin = (Pm + (Gm << 1)) ^ Pm;
    sub_word<M>(d, (uint32_t)(bin >> g.t) & 1u);
    const uint32_t borrow_out = (uint32_t)(bin >> G) & 1u;
    const uint32_t ge = carry | (borrow_out ^ 1u);
    const uint32_t msk = 0u - ge;
#pragma unroll
    for (int j = 0; j < M; ++j) c[j] = (d[j] & msk) | (c[j] & ~msk);
    g.sync();
    sts<M>(OUT + g.t * M, c);
    g.sync();
}

// Steps of a Montgomery product. The kernels call the product from exactly one
// place (a loop over the products of the job), so each step exists once in the
// instruction stream although it is inlined.
template <class S>
MPG_DI void step_mul(Grp<S> g) { phase_mul<S>(g, g.X(), g.Y(), g.T()); }

template <class S>
MPG_DI void step_sqr(Grp<S> g) { phase_sqr<S>(g, g.X(), g.X(), g.T()); }   // squares in X, Y

// T (2*NP words) -> X = T * R^-1 mod N (q goes to Y). RED: 0 truncated (Alg. 6), 1 classical (Alg. 5).
// lazy: no final subtraction; with 4N <= R and T < 4N^2 the result stays below 2N (the slack
// that lets the paper's Alg. 3 and Alg. 5 skip it).
// c_add = [T mod R != 0] and low_zero = [T mod W^(NP-1) == 0], for the whole group
template <class S>
MPG_DI void reduce_flags(const Grp<S> &g, const uint32_t *T, uint32_t &c_add, uint32_t &low_zero) {
    constexpr int M = S::M, NP = S::NP;
    uint32_t nz_all = 0u, nz_low = 0u;
    {
        uint32_t x[M];
        lds<M>(x, T + g.t * M);
#pragma unroll
        for (int j = 0; j < M; ++j) {
            nz_all |= x[j];
            if (g.t * M + j < NP - 1) nz_low |= x[j];
        }
    }
    const bool pr[2] = {nz_all != 0u, nz_low != 0u};
    uint32_t mk[2];
    g.template bits<2>(pr, mk);
    c_add = mk[0] ? 1u : 0u;
    low_zero = mk[1] ? 0u : 1u;
}

template <class S, int RED>
MPG_DI void step_reduce(Grp<S> g, bool lazy) {
    constexpr int M = S::M, NP = S::NP;
    uint32_t *T = g.T();
    uint32_t c_add, low_zero;
    reduce_flags<S>(g, T, c_add, low_zero);
    phase_mullo<S>(g, T, g.NI(), g.Q());
    if constexpr (RED == 0) {
        const uint32_t carry = phase_mulhi<S>(g, g.Q(), g.N(), T, c_add, low_zero, g.X());
        if (!lazy) cond_sub<S>(g, g.X(), carry, g.N(), g.X());
    } else {
        (void)c_add;
        (void)low_zero;
        const uint32_t carry = phase_fma<S>(g, g.Q(), g.N(), T);
        if (!lazy) {
            cond_sub<S>(g, T + NP, carry, g.N(), g.X());
        } else {
            uint32_t x[M];
            lds<M>(x, T + NP + g.t * M);
            sts<M>(g.X() + g.t * M, x);
            g.sync();
        }
    }
}

// ------------------------------------------------------------------ CIOS (Alg. 4)
//
// Word-serial Montgomery product (the paper's CIOS-inspired batch algorithm): for each
// word a_i of X, Y += a_i * B, q = (Y mod W) * n0' mod W, Y = (Y + q * N) / W. Thread t
// keeps words tM .. tM+M-1 of Y plus two carry-save words above them (positions
// (t+1)M and (t+1)M+1, which overlap the next thread's words), so a step needs no
// carry propagation across threads: the division by W moves every word down one place
// and thread t+1's lowest word joins thread t's word M-1. The carry-save sum stays
// below 3 W^(M+1) per thread. Inter-thread carries are resolved once at the end.
// Rotation: in step s of a body, logical word j of the thread's M+2 words sits in
// register (j + s) mod (M+2), so the shift costs no register moves; a body of M+2 steps
// brings the rotation back to 0.

// logical y[0 .. M+1] += x * v[0 .. M-1] (rotation R)
template <int M, int R>
MPG_DI void cios_rowmac(uint32_t (&y)[M + 2], uint32_t x, const uint32_t (&v)[M]) {
    constexpr int L = M + 2;
    mad_lo_cc(y[R % L], x, v[0]);
    madc_hi_cc(y[(1 + R) % L], x, v[0]);
#pragma unroll
    for (int j = 2; j < M; j += 2) {
        madc_lo_cc(y[(j + R) % L], x, v[j]);
        madc_hi_cc(y[(j + 1 + R) % L], x, v[j]);
    }
    addc_cc(y[(M + R) % L], 0u);
    addc(y[(M + 1 + R) % L], 0u);
    mad_lo_cc(y[(1 + R) % L], x, v[1]);
    madc_hi_cc(y[(2 + R) % L], x, v[1]);
#pragma unroll
    for (int j = 3; j < M; j += 2) {
        madc_lo_cc(y[(j + R) % L], x, v[j]);
        madc_hi_cc(y[(j + 1 + R) % L], x, v[j]);
    }
    addc(y[(M + 1 + R) % L], 0u);
}

// CNT steps starting at word i of X, the first with rotation R
template <class S, int R, int CNT>
MPG_DI void cios_steps(const Grp<S> &g, uint32_t (&y)[S::M + 2], int i, const uint32_t (&b)[S::M],
                       const uint32_t (&nn)[S::M], uint32_t n0i) {
    if constexpr (CNT > 0) {
        constexpr int M = S::M, L = M + 2, G = S::G;
        const uint32_t a = g.X()[i];
        cios_rowmac<M, R>(y, a, b);
        const uint32_t q = __shfl_sync(0xffffffffu, y[R % L], g.gbase) * n0i;   // word 0 is thread 0's
        cios_rowmac<M, R>(y, q, nn);
        const uint32_t z = __shfl_sync(0xffffffffu, y[R % L], g.gbase + (g.t + 1 < G ? g.t + 1 : 0));
        y[R % L] = 0u;   // word 0 leaves; this register becomes logical word M+1
        constexpr int R1 = (R + 1) % L;
        add_cc(y[(M - 1 + R1) % L], g.t + 1 < G ? z : 0u);
        addc_cc(y[(M + R1) % L], 0u);
        addc(y[(M + 1 + R1) % L], 0u);
        cios_steps<S, R1, CNT - 1>(g, y, i + 1, b, nn, n0i);
    }
}

// X <- X * Y * W^-NP (< 2N for inputs < 2N when 4N <= W^NP), returns the word above X
template <class S>
MPG_DI uint32_t cios_product(const Grp<S> &g, bool square) {
    constexpr int G = S::G, M = S::M, NP = S::NP, L = M + 2;
    static_assert(M % 2 == 0 && M >= 4, "CIOS needs an even M >= 4");
    static_assert(!S::WMAP, "CIOS passes a word between threads at every step: lane mapping only");
    uint32_t b[M], nn[M], y[L];
    lds<M>(b, (square ? g.X() : g.Y()) + g.t * M);
    lds<M>(nn, g.N() + g.t * M);
    const uint32_t n0i = g.NI()[0];   // N' mod W = (-N)^-1 mod W
    zero<L>(y);
    constexpr int BODIES = NP / L, REM = NP % L;
    MPG_BLOCK_LOOP
    for (int k = 0; k < BODIES; ++k) cios_steps<S, 0, L>(g, y, k * L, b, nn, n0i);
    cios_steps<S, 0, REM>(g, y, BODIES * L, b, nn, n0i);
    // resolve the carry-save words: thread t-1's two top words sit on this thread's words 0, 1
    uint32_t lo[M];
#pragma unroll
    for (int j = 0; j < M; ++j) lo[j] = y[(j + REM) % L];
    const uint32_t o0 = y[(M + REM) % L], o1 = y[(M + 1 + REM) % L];
    const int src = g.gbase + (g.t > 0 ? g.t - 1 : 0);
    const uint32_t i0 = __shfl_sync(0xffffffffu, o0, src), i1 = __shfl_sync(0xffffffffu, o1, src);
    add_cc(lo[0], g.t > 0 ? i0 : 0u);
    addc_cc(lo[1], g.t > 0 ? i1 : 0u);
#pragma unroll
    for (int j = 2; j < M; ++j) addc_cc(lo[j], 0u);
    const uint32_t cgen = addc_get();
    uint32_t all = lo[0];
#pragma unroll
    for (int j = 1; j < M; ++j) all &= lo[j];
    const uint64_t Gm = g.gbits(cgen != 0u), Pm = g.gbits(all == 0xffffffffu);
    const uint64_t cin = (Pm + (Gm << 1)) ^ Pm;
    add_word<M>(lo, (uint32_t)(cin >> g.t) & 1u);
    const uint32_t top = __shfl_sync(0xffffffffu, o0, g.gbase + G - 1) + ((uint32_t)(cin >> G) & 1u);
    gsync();   // every thread has read X
    sts<M>(g.X() + g.t * M, lo);
    gsync();
    return top;
}

template <class S>
MPG_DI void step_cios(const Grp<S> &g, bool square, bool lazy) {
    const uint32_t top = cios_product<S>(g, square);
    if (!lazy) cond_sub<S>(g, g.X(), top, g.N(), g.X());
}

// Montgomery product with one Karatsuba level and the Karatsuba form of the truncated
// reduction (mp_tkara.cuh), for its own layouts (KShape).
template <class S>
MPG_DI void tk_prepare(const Grp<S> &g);
template <class S>
MPG_DI void tk_product(const Grp<S> &g, bool square, bool lazy);

// once per kernel, after N and N' are in shared memory (and synchronised): per-modulus
// values that the products of reduction RED reuse
template <class S, int RED>
MPG_DI void mont_prepare(const Grp<S> &g) {
    if constexpr (RED == 3) tk_prepare<S>(g);
}

// X <- X * Y * R^-1 mod N (or X^2 * R^-1 when square): X, Y, N, N' in shared memory.
// Y is overwritten (it holds q afterwards). RED: 0 truncated (Alg. 6), 1 classical (Alg. 5),
// 2 word-serial CIOS (Alg. 4), 3 truncated in its Karatsuba form (Sec. 5.1; KShape layouts).
template <class S, int RED>
MPG_DI void mont_mul(const Grp<S> &g, bool square, bool lazy) {
    if constexpr (RED == 3) {
        tk_product<S>(g, square, lazy);
    } else if constexpr (RED == 2) {
        step_cios<S>(g, square, lazy);
    } else {
        if (square) step_sqr<S>(g);
        else step_mul<S>(g);
        step_reduce<S, RED>(g, lazy);
    }
}

}  // namespace mpg
