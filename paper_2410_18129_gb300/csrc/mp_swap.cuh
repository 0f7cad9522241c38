// Role-swapped groups for the Montgomery kernels of the block-product reductions
// (truncated, Alg. 6; classical, Alg. 3/5).
//
// A block holds 32 instances in G warps and every instance keeps one record of shared
// memory, as in mp_group.cuh. The same records are worked on under two thread mappings:
//   * product view: warp t plays thread t of all 32 instances (lane = instance). The block
//     products of a phase then run with a warp-uniform thread index: each slot gets its own
//     loop of exactly its block count, and a slot is stored when its loop ends (no
//     thread-dependent slot switch inside a loop). Global loads and stores of an instance's
//     words (operands, context, window-table scans) are coalesced across the 32 instances.
//   * carry view: the G threads of an instance are G consecutive lanes of one warp (32/G
//     instances per warp). Carry resolution, the c_add / low-zero tests, the group sum of
//     the Thm. 2 boundary terms and the final subtraction use shuffles and ballots there;
//     each phase's resolve keeps its final words in registers, derives the flags or does the
//     constant-time subtraction on them, and stores once.
// A block barrier separates the two views; a Montgomery product crosses six of them.
// T and the slot spill area are padded with four words after every 32: a carry-view thread
// reads its M-word slots at stride M, and without the pad lanes t and t+4 of an instance
// (M = 8) or lanes t, t+2, ... (M = 16) hit the same banks.
#pragma once
#include "mp_kernels.cuh"

namespace mpg {

// word offset of logical word i of a padded array (T, slot spills): four pad words follow
// every 32 words. Blocks of 4, 8 or 16 words never straddle a row, so they stay contiguous.
// Shapes whose M is not a multiple of 8 do not pad (P = false).
template <bool P = true>
MPG_DI int pad32(int i) { return P ? i + ((i >> 5) << 2) : i; }
constexpr int pad_size(int n, bool p = true) { return !p ? n : n ? (n - 1) + (((n - 1) >> 5) << 2) + 1 : 0; }
constexpr int pad_index(int i, bool p = true) { return p ? i + ((i >> 5) << 2) : i; }

template <bool P>
struct PadMap {
    MPG_DI int operator()(int i) const { return pad32<P>(i); }
};

template <int G_, int M_>
struct Swap {
    using PS = Shape<G_, M_, true>;    // product view
    using LS = Shape<G_, M_, false>;   // carry view
    static constexpr int G = G_, M = M_, NP = G_ * M_, H = M_ / 2;
    static constexpr int TPB = 32 * G_;   // 32 instances per block
    static_assert(LS::MONT_OK, "Montgomery needs an even M >= 4");
    static_assert(PS::OFF_T == LS::OFF_T, "one record layout for both views");
    static_assert(32 % G_ == 0, "the G threads of an instance share a warp in the carry view");
    // pad T and the spills where a thread's M-word slots repeat the bank pattern (M = 8, 16)
    static constexpr bool PAD = (M_ % 8 == 0);
    // record: X, Y (q), N, N' (NP words each), T (2NP, padded), spills: hi words of 2G slots of
    // up to M words (padded), then one top word per slot
    static constexpr int OFF_T = LS::OFF_T;
    static constexpr int OFF_P = (OFF_T + pad_size(2 * NP, PAD) + 3) & ~3;
    static constexpr int SPILL_TOP = (pad_size(2 * G * M, PAD) + 3) & ~3;
    // one word: ((-T) mod R)[NP-1] for the carry recovery of the truncated high half (Thm. 1/2)
    static constexpr int OFF_L = OFF_P + SPILL_TOP + 2 * G;
    static constexpr int WORDS_RAW = OFF_L + 1;
    // Thm. 2 boundary sums exchanged through T's low half (dead once q is formed): ZW words per
    // thread at padded offsets, 16-byte aligned
    static constexpr int ZW = (H + 3 + 3) & ~3;
    static_assert(pad_index((G - 1) * ZW, PAD) + ZW <= pad_index(NP, PAD), "Z exchange must stay below T's high half");
    // product view: the 32 lanes of a warp read the same offset of 32 records; a stride of
    // 4 (mod 8) words puts each group of 8 lanes' 16-byte accesses on distinct banks
    static constexpr int WORDS = ((WORDS_RAW + 3) / 8) * 8 + 4;
    static constexpr size_t SMEM = (size_t)32 * WORDS * 4;
};

template <class W>
struct Views {
    Grp<typename W::PS> p;   // product view
    Grp<typename W::LS> l;   // carry view
};

template <class W>
MPG_DI Views<W> swap_views(uint32_t *smem) {
    Views<W> v;
    const int lane = (int)(threadIdx.x & 31), warp = (int)(threadIdx.x >> 5);
    v.p.sm = smem + lane * W::WORDS;
    v.p.pa = v.p.sm + W::OFF_P;
    v.p.t = warp;
    v.p.gbase = 0;
    const int li = warp * (32 / W::G) + lane / W::G;
    v.l.sm = smem + li * W::WORDS;
    v.l.pa = v.l.sm + W::OFF_P;
    v.l.t = lane % W::G;
    v.l.gbase = lane & ~(W::G - 1);
    return v;
}

// instance of the product view in the launch
MPG_DI size_t swap_instance() { return (size_t)blockIdx.x * 32 + (threadIdx.x & 31); }

MPG_DI void bsync() { __syncthreads(); }

// Spill of slot s for B-word slots: its hi words B .. 2B-1 at P + pad32(s*B); its top word 2B
// beside the top of the other slot of the same thread of the product view, so that the two go
// out in one 8-byte store: entry top_index(s) of the 2G words at P + SPILL_TOP.
template <class W, int B, class S>
MPG_DI uint32_t *swp_hi(const Grp<S> &g, int s) { return g.P() + pad32<W::PAD>(s * B); }

template <int G, int PAT>
MPG_DI int top_index(int s) {
    if constexpr (PAT == PAT_SEQ) return 2 * (s % G) + s / G;     // thread s mod G: slots t, G+t
    else return s < G ? 2 * s : 2 * (2 * G - 1 - s) + 1;          // zigzag: slots t, 2G-1-t
}

// store the low and hi words of a slot sum; returns its top word (word 2B; word 2B+1 is zero)
template <int B>
MPG_DI uint32_t store_lohi(const uint32_t (&V)[2 * B + 2], uint32_t *out_lo, uint32_t *out_hi) {
    uint32_t lo[B], hi[B];
#pragma unroll
    for (int j = 0; j < B; ++j) { lo[j] = V[j]; hi[j] = V[B + j]; }
    sts<B>(out_lo, lo);
    sts<B>(out_hi, hi);
    return V[2 * B];
}

// the top words of this thread's first and second slot
template <class W, class S>
MPG_DI void store_tops(const Grp<S> &g, uint32_t top0, uint32_t top1) {
    *reinterpret_cast<uint2 *>(g.P() + W::SPILL_TOP + 2 * g.t) = make_uint2(top0, top1);
}

// ------------------------------------------------------------------ product-view phases
//
// Thread t of every instance is warp t here, so each slot's blocks form one run of mac_run
// with a warp-uniform count, and a slot is stored straight after its run.

// slot sums of T = X * Y: thread t owns slots t (X_j Y_{t-j}, j <= t) and G+t (j > t)
template <class W>
MPG_DI void swp_mul_slots(const Grp<typename W::PS> &g, const uint32_t *X, const uint32_t *Y, uint32_t *T) {
    constexpr int G = W::G, M = W::M, U = run_group<M>();
    const int t = g.t;
    Acc3<M> a;
    uint32_t V[2 * M + 2];
    acc3_zero<M>(a);
    mac_run<M, U>(a, X, Y, t + 1, [&](int j, int &u, int &v) { u = j; v = t - j; });
    acc3_value<M>(V, a);
    const uint32_t top0 = store_lohi<M>(V, T + pad32<W::PAD>(t * M), swp_hi<W, M>(g, t));
    acc3_zero<M>(a);
    mac_run<M, U>(a, X, Y, G - 1 - t, [&](int j, int &u, int &v) { u = t + 1 + j; v = G - 1 - j; });
    acc3_value<M>(V, a);
    const uint32_t top1 = store_lohi<M>(V, T + pad32<W::PAD>((G + t) * M), swp_hi<W, M>(g, G + t));
    store_tops<W>(g, top0, top1);
}

// V (2M+2 words, below W^(2M+1) / 2) <- 2 V + the squares x_i^2 at columns 2i
template <int M>
MPG_DI void double_add_diag(uint32_t (&V)[2 * M + 2], const uint32_t (&x)[M]) {
#pragma unroll
    for (int k = 2 * M + 1; k > 0; --k) V[k] = __funnelshift_l(V[k - 1], V[k], 1);
    V[0] <<= 1;
    mad_lo_cc(V[0], x[0], x[0]);
    madc_hi_cc(V[1], x[0], x[0]);
#pragma unroll
    for (int i = 1; i < M; ++i) {
        madc_lo_cc(V[2 * i], x[i], x[i]);
        madc_hi_cc(V[2 * i + 1], x[i], x[i]);
    }
    addc_cc(V[2 * M], 0u);
    addc(V[2 * M + 1], 0u);
}

// Slot sums of T = X^2, complete (no transform left for the resolve). Thread t owns slots t
// and G+t (the cross products X_u X_v, u < v, on those diagonals). The square of block u
// covers exactly the columns of slot 2u, so the owner of an even slot s (an even t: both of
// its slots are even) adds X_{s/2}^2 itself: the block's cross terms join the accumulator
// before the doubling, its squares x_i^2 after it. Every slot sum stays below
// (G + 2) W^(2M) < W^(2M+1).
template <class W>
MPG_DI void swp_sqr_slots(const Grp<typename W::PS> &g, const uint32_t *X, uint32_t *T) {
    constexpr int G = W::G, M = W::M, U = run_group<M>();
    const int t = g.t;
    const bool even = (t & 1) == 0;
    const int nA = (t + 1) >> 1;              // pairs u < v with u + v = t
    const int nB = ((G - t + 1) >> 1) - 1;    // pairs with u + v = G + t
    Acc3<M> a;
    uint32_t top[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int s = k ? G + t : t;
        acc3_zero<M>(a);
        if (k == 0) mac_run<M, U>(a, X, X, nA, [&](int j, int &u, int &v) { u = j; v = t - j; });
        else mac_run<M, U>(a, X, X, nB, [&](int j, int &u, int &v) { u = t + 1 + j; v = G - 1 - j; });
        uint32_t x[M];
        if (even) {   // warp-uniform
            lds<M>(x, X + (s >> 1) * M);
            acc3_tri<M>(a, x);
        } else {
            zero<M>(x);
        }
        uint32_t V[2 * M + 2];
        acc3_value<M>(V, a);
        double_add_diag<M>(V, x);
        top[k] = store_lohi<M>(V, T + pad32<W::PAD>(s * M), swp_hi<W, M>(g, s));
    }
    store_tops<W>(g, top[0], top[1]);
}

// slot sums of q = T_lo * N' mod R in H-word slots: thread t owns slots t (t+1 blocks) and
// 2G-1-t (2G-t blocks); T is read through its padding
template <class W>
MPG_DI void swp_mullo_slots(const Grp<typename W::PS> &g, const uint32_t *T, const uint32_t *NI, uint32_t *Q) {
    constexpr int G = W::G, H = W::H, U = run_group<H>();
    const int t = g.t;
    Acc3<H> a;
    uint32_t V[2 * H + 2];
    acc3_zero<H>(a);
    mac_run<H, U>(a, T, NI, t + 1, [&](int j, int &u, int &v) { u = j; v = t - j; }, PadMap<W::PAD>{});
    acc3_value<H>(V, a);
    const uint32_t top0 = store_lohi<H>(V, Q + t * H, swp_hi<W, H>(g, t));
    acc3_zero<H>(a);
    mac_run<H, U>(a, T, NI, 2 * G - t, [&](int j, int &u, int &v) { u = j; v = 2 * G - 1 - t - j; }, PadMap<W::PAD>{});
    acc3_value<H>(V, a);
    const uint32_t top1 = store_lohi<H>(V, Q + (2 * G - 1 - t) * H, swp_hi<W, H>(g, 2 * G - 1 - t));
    store_tops<W>(g, top0, top1);
}

// slot sums of the classical reduction T + q*N over all 2*NP words: T's words of a slot are
// added before the slot is stored over them
template <class W>
MPG_DI void swp_fma_slots(const Grp<typename W::PS> &g, const uint32_t *Qs, const uint32_t *Ns, uint32_t *T) {
    constexpr int G = W::G, M = W::M, U = run_group<M>();
    const int t = g.t;
    Acc3<M> a;
    uint32_t top[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int s = k ? G + t : t;
        acc3_zero<M>(a);
        if (k == 0) mac_run<M, U>(a, Qs, Ns, t + 1, [&](int j, int &u, int &v) { u = j; v = t - j; });
        else mac_run<M, U>(a, Qs, Ns, G - 1 - t, [&](int j, int &u, int &v) { u = t + 1 + j; v = G - 1 - j; });
        uint32_t V[2 * M + 2], d[M];
        acc3_value<M>(V, a);
        lds<M>(d, T + pad32<W::PAD>(s * M));
        add_cc(V[0], d[0]);
#pragma unroll
        for (int j = 1; j < M; ++j) addc_cc(V[j], d[j]);
#pragma unroll
        for (int j = M; j < 2 * M + 1; ++j) addc_cc(V[j], 0u);
        addc(V[2 * M + 1], 0u);
        top[k] = store_lohi<M>(V, T + pad32<W::PAD>(s * M), swp_hi<W, M>(g, s));
    }
    store_tops<W>(g, top[0], top[1]);
}

// Boundary terms of Thm. 2 for one H x H block product X*Y on the diagonal u + v = 2G-1, whose
// local column c = i+j sits at global column NP-H+c; Z word 0 is column NP-1. Needed: the
// pairs with c >= H-1 in full (Z words c-H+1, c-H+2) and the hi halves of the pairs with
// c = H-2 (Z word 0). In row i the pairs c >= H-1 are j = H-1-i .. H-1: a chain over every
// other j starts at Z word 0 (pairs at even words, ZE) and one at Z word 1 (odd words, ZO,
// ZO[k] = word k+1); their carries go to counters ZK. The hi halves go to the two-word zh.
template <int H>
struct ZAcc {
    static constexpr int LE = (H + 2) & ~1;   // even pairs up to word H
    uint32_t E[LE];
    uint32_t O[LE];
    uint32_t K[H + 3];
    uint32_t h0, h1;
};

template <int H, int I>
MPG_DI void zacc_row(ZAcc<H> &z, uint32_t xi, const uint32_t (&y)[H]) {
    constexpr int J0A = H - 1 - I, NA = I / 2 + 1;   // chain A: j = H-1-I, H+1-I, ...
    acc3_chain<H, ZAcc<H>::LE, J0A, 0, NA>(z.E, z.K[2 * NA], xi, y);
    if constexpr (I >= 1) {
        constexpr int J0B = H - I, NB = (I - 1) / 2 + 1;   // chain B: j = H-I, H-I+2, ...
        acc3_chain<H, ZAcc<H>::LE, J0B, 0, NB>(z.O, z.K[2 * NB + 1], xi, y);
    }
    if constexpr (I <= H - 2) {   // hi half of x_I * y_{H-2-I} (column H-2)
        mad_hi_cc(z.h0, xi, y[H - 2 - I]);
        addc(z.h1, 0u);
    }
}

template <int H, int I = 0>
MPG_DI void zacc_rows(ZAcc<H> &z, const uint32_t (&x)[H], const uint32_t (&y)[H]) {
    if constexpr (I < H) {
        zacc_row<H, I>(z, x[I], y);
        zacc_rows<H, I + 1>(z, x, y);
    }
}

// Z[0 .. H+3) = value of z
template <int H>
MPG_DI void zacc_value(uint32_t (&Z)[H + 3], const ZAcc<H> &z) {
    constexpr int LE = ZAcc<H>::LE;
#pragma unroll
    for (int k = 0; k < H + 3; ++k) Z[k] = k < LE ? z.E[k] : 0u;
    add_cc(Z[1], z.O[0]);
#pragma unroll
    for (int k = 1; k < LE && k + 1 < H + 3; ++k) addc_cc(Z[k + 1], z.O[k]);
#pragma unroll
    for (int k = LE + 1; k < H + 3; ++k) addc_cc(Z[k], 0u);
    add_cc(Z[0], z.h0);
    addc_cc(Z[1], z.h1);
#pragma unroll
    for (int k = 2; k < H + 3; ++k) addc_cc(Z[k], z.K[k]);
}

// Slot sums of the truncated high half C = floor(T/R) + floor(qN/R) (Alg. 6) in the product
// view: the block products of qN with u + v >= 2G in H-word slots (thread t: slots t and
// 2G-1-t), T's high words of each slot added before it is stored, and this thread's share
// of the Thm. 2 boundary sum parked in T's low half (dead once q is formed; word NP-1 kept).
template <class W>
MPG_DI void swp_mulhi_slots(const Grp<typename W::PS> &g, const uint32_t *Qs, const uint32_t *Ns, uint32_t *C,
                            const uint32_t *T) {
    constexpr int G = W::G, H = W::H, NP = W::NP;
    const int t = g.t;
    {
        ZAcc<H> z;
        zero<ZAcc<H>::LE>(z.E);
        zero<ZAcc<H>::LE>(z.O);
        zero<H + 3>(z.K);
        z.h0 = 0u;
        z.h1 = 0u;
#pragma unroll
        for (int j = 0; j < 2; ++j) {   // boundary terms of the diagonal blocks u + v = 2G-1
            const int u = 2 * t + j;
            uint32_t x[H], y[H];
            lds<H>(x, Qs + u * H);
            lds<H>(y, Ns + (2 * G - 1 - u) * H);
            zacc_rows<H>(z, x, y);
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {   // corner hi halves of the blocks u + v = 2G-2
            const int u = 2 * t + j;
            const bool live = u <= 2 * G - 2;
            const uint32_t xq = Qs[u * H + H - 1];
            const uint32_t yn = live ? Ns[(2 * G - 2 - u) * H + H - 1] : 0u;
            mad_hi_cc(z.h0, xq, yn);
            addc(z.h1, 0u);
        }
        uint32_t Z[H + 3], Zs[W::ZW];
        zacc_value<H>(Z, z);
#pragma unroll
        for (int k = 0; k < W::ZW; ++k) Zs[k] = k < H + 3 ? Z[k] : 0u;
        sts<W::ZW>(g.T() + pad32<W::PAD>(t * W::ZW), Zs);
    }
    constexpr int U = run_group<H>();
    Acc3<H> a;
    uint32_t top[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int s = k ? 2 * G - 1 - t : t;
        acc3_zero<H>(a);
        if (k == 0) mac_run<H, U>(a, Qs, Ns, 2 * G - 1 - t, [&](int j, int &u, int &v) { u = t + 1 + j; v = 2 * G - 1 - j; });
        else mac_run<H, U>(a, Qs, Ns, t, [&](int j, int &u, int &v) { u = 2 * G - t + j; v = 2 * G - 1 - j; });
        uint32_t V[2 * H + 2], d[H];
        acc3_value<H>(V, a);
        lds<H>(d, T + pad32<W::PAD>(NP + s * H));
        add_cc(V[0], d[0]);
#pragma unroll
        for (int j = 1; j < H; ++j) addc_cc(V[j], d[j]);
#pragma unroll
        for (int j = H; j < 2 * H + 1; ++j) addc_cc(V[j], 0u);
        addc(V[2 * H + 1], 0u);
        top[k] = store_lohi<H>(V, C + s * H, swp_hi<W, H>(g, s));
    }
    store_tops<W>(g, top[0], top[1]);
}

// ------------------------------------------------------------------ carry-view phases

// Resolve the stored slot sums (low words at OUT through om, spills in the padded area) into
// final words: add each predecessor's spill, pass the overflow word on with a shuffle, and
// resolve the remaining one-bit carries of the group with ballots (carry-lookahead). The
// final words of this thread's two slots are left in fin[k] (slot slot_of<G, PAT>(t, k)),
// not stored; only their owner reads a slot's low words, so the caller may store them at
// once. Returns the low word of everything above the last slot.
template <class W, int B, int PAT, class OM>
MPG_DI uint32_t cv_resolve(const Grp<typename W::LS> &g, const uint32_t (&in0)[B + 2], const uint32_t *OUT, const OM &om,
                           uint32_t (&fin)[2][B]) {
    constexpr int G = W::G, NSLOT = 2 * G;
    uint32_t top = 0u;
    uint32_t ov[2][2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int s = slot_of<G, PAT>(g.t, k);
        uint32_t lo[B];
        lds<B>(lo, OUT + om(s * B));
        if (s == NSLOT - 1) top = g.P()[pad32<W::PAD>(s * B)];   // word B of the last slot's sum
        uint32_t x[B + 2];
        if (s == 0) {
#pragma unroll
            for (int j = 0; j < B + 2; ++j) x[j] = in0[j];
        } else {
            uint32_t h[B];
            lds<B>(h, g.P() + pad32<W::PAD>((s - 1) * B));
#pragma unroll
            for (int j = 0; j < B; ++j) x[j] = h[j];
            x[B] = g.P()[W::SPILL_TOP + top_index<G, PAT>(s - 1)];
            x[B + 1] = 0u;
        }
        add_cc(x[0], lo[0]);
#pragma unroll
        for (int j = 1; j < B; ++j) addc_cc(x[j], lo[j]);
        addc_cc(x[B], 0u);
        addc(x[B + 1], 0u);
#pragma unroll
        for (int j = 0; j < B; ++j) fin[k][j] = x[j];
        ov[k][0] = x[B];
        ov[k][1] = x[B + 1];
        if (s == NSLOT - 1) top += x[B];
    }
    uint32_t oin[2][2];
    pred_overflow<G, PAT>(g.t, g.gbase, ov[0], ov[1], oin[0], oin[1]);
    uint32_t cgen[2], cprop[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        add_cc(fin[k][0], oin[k][0]);
        addc_cc(fin[k][1], oin[k][1]);
#pragma unroll
        for (int j = 2; j < B; ++j) addc_cc(fin[k][j], 0u);
        cgen[k] = addc_get();
        uint32_t all = fin[k][0];
#pragma unroll
        for (int j = 1; j < B; ++j) all &= fin[k][j];
        cprop[k] = (all == 0xffffffffu) ? 1u : 0u;
    }
    const bool pr[4] = {cgen[0] != 0u, cprop[0] != 0u, cgen[1] != 0u, cprop[1] != 0u};
    uint32_t mk[4];
    g.template bits<4>(pr, mk);
    const uint64_t Gm = slot_mask<G, PAT>(mk[0], mk[2]);
    const uint64_t Pm = slot_mask<G, PAT>(mk[1], mk[3]);
    const uint64_t cin = (Pm + (Gm << 1)) ^ Pm;
#pragma unroll
    for (int k = 0; k < 2; ++k) add_word<B>(fin[k], (uint32_t)(cin >> slot_of<G, PAT>(g.t, k)) & 1u);
    constexpr int owner = (PAT == PAT_ZIGZAG) ? 0 : G - 1;
    top = g.bcast(top, owner);
    return top + ((uint32_t)(cin >> NSLOT) & 1u);
}

// T resolved in place, and c_add = [T mod R != 0], low_zero = [T mod W^(NP-1) == 0] for the
// whole group from the resolved words (slot t, this thread's first, is T's words tM..tM+M-1)
template <class W>
MPG_DI void cv_resolve_T(const Grp<typename W::LS> &g, uint32_t &c_add, uint32_t &low_zero) {
    constexpr int M = W::M, NP = W::NP, G = W::G;
    uint32_t in0[M + 2], fin[2][M];
    zero<M + 2>(in0);
    cv_resolve<W, M, PAT_SEQ>(g, in0, g.T(), PadMap<W::PAD>{}, fin);
    uint32_t nz_all = 0u, nz_low = 0u;
#pragma unroll
    for (int j = 0; j < M; ++j) {
        nz_all |= fin[0][j];
        if (g.t * M + j < NP - 1) nz_low |= fin[0][j];
    }
    const bool pr[2] = {nz_all != 0u, nz_low != 0u};
    uint32_t mk[2];
    g.template bits<2>(pr, mk);
    c_add = mk[0] ? 1u : 0u;
    low_zero = mk[1] ? 0u : 1u;
    // ((-T) mod R)[NP-1] = ~T[NP-1] + [T[0 .. NP-1) == 0]  (mod W); word NP-1 is the last word of
    // slot G-1
    if (g.t == G - 1) g.sm[W::OFF_L] = ~fin[0][M - 1] + low_zero;
    sts<M>(g.T() + pad32<W::PAD>(g.t * M), fin[0]);
    sts<M>(g.T() + pad32<W::PAD>((G + g.t) * M), fin[1]);
}

// q resolved in place (H-word slots in Y)
template <class W>
MPG_DI void cv_resolve_q(const Grp<typename W::LS> &g) {
    constexpr int H = W::H, G = W::G;
    uint32_t in0[H + 2], fin[2][H];
    zero<H + 2>(in0);
    cv_resolve<W, H, PAT_ZIGZAG>(g, in0, g.Q(), IdMap{}, fin);
    sts<H>(g.Q() + g.t * H, fin[0]);
    sts<H>(g.Q() + (2 * G - 1 - g.t) * H, fin[1]);
}

// OUT segments = (top*R + C >= N) ? C - N : C, constant time, for two segments per thread of
// K words in slot order PAT; borrows cross the group with the same lookahead as carries
template <class W, int K, int PAT>
MPG_DI void cv_cond_sub(const Grp<typename W::LS> &g, uint32_t (&c)[2][K], uint32_t top, const uint32_t *Ns, uint32_t *OUT) {
    constexpr int G = W::G, NSEG = (PAT == PAT_ONE) ? G : 2 * G;
    constexpr int NK = (PAT == PAT_ONE) ? 1 : 2;
    uint32_t d[2][K];
    bool pr[4] = {false, false, false, false};
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const int s = slot_of<G, PAT>(g.t, k);
        uint32_t n[K];
        lds<K>(n, Ns + s * K);
        uint32_t eq = 0u;
#pragma unroll
        for (int j = 0; j < K; ++j) { d[k][j] = c[k][j]; eq |= c[k][j] ^ n[j]; }
        pr[2 * k] = sub_n<K>(d[k], n) != 0u;
        pr[2 * k + 1] = eq == 0u;
    }
    uint32_t mk[4];
    g.template bits<4>(pr, mk);
    const uint64_t Gm = slot_mask<G, PAT>(mk[0], mk[2]);
    const uint64_t Pm = slot_mask<G, PAT>(mk[1], mk[3]);
    const uint64_t bin = (Pm + (Gm << 1)) ^ Pm;
    const uint32_t borrow_out = (uint32_t)(bin >> NSEG) & 1u;
    const uint32_t msk = 0u - (top | (borrow_out ^ 1u));
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const int s = slot_of<G, PAT>(g.t, k);
        sub_word<K>(d[k], (uint32_t)(bin >> s) & 1u);
#pragma unroll
        for (int j = 0; j < K; ++j) d[k][j] = (d[k][j] & msk) | (c[k][j] & ~msk);
        sts<K>(OUT + s * K, d[k]);
    }
}

// truncated high half: group sum of the boundary terms, carry recovery from word NP-1 of -T
// (Thm. 1/2), C = floor(T/R) + floor(qN/R) + c_add resolved, then the final subtraction on the
// resolved words (skipped when lazy); result in X
template <class W>
MPG_DI void cv_resolve_hi(const Grp<typename W::LS> &g, uint32_t c_add, uint32_t low_zero, bool lazy) {
    constexpr int H = W::H, G = W::G;
    uint32_t Z[H + 3];
    {
        uint32_t Zs[W::ZW];
        lds<W::ZW>(Zs, g.T() + pad32<W::PAD>(g.t * W::ZW));
#pragma unroll
        for (int k = 0; k < H + 3; ++k) Z[k] = Zs[k];
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {   // sum over the instance's G lanes
        uint32_t o[H + 3];
#pragma unroll
        for (int k = 0; k < H + 3; ++k) o[k] = __shfl_xor_sync(0xffffffffu, Z[k], off);
        add_n<H + 3>(Z, o);
    }
    (void)low_zero;
    const uint32_t L = g.sm[W::OFF_L];   // ((-T) mod R)[NP-1], saved by cv_resolve_T
    const uint32_t extra = (uint32_t)(((uint64_t)L - (uint64_t)Z[0]) >> 63);   // [L < Z[0]]
    uint32_t in0[H + 2], fin[2][H];
#pragma unroll
    for (int j = 0; j < H + 2; ++j) in0[j] = Z[1 + j];
    add_word<H + 2>(in0, extra + c_add);
    const uint32_t top = cv_resolve<W, H, PAT_ZIGZAG>(g, in0, g.X(), IdMap{}, fin);
    if (lazy) {
        sts<H>(g.X() + g.t * H, fin[0]);
        sts<H>(g.X() + (2 * G - 1 - g.t) * H, fin[1]);
    } else {
        cv_cond_sub<W, H, PAT_ZIGZAG>(g, fin, top, g.N(), g.X());
    }
}

// classical: T + qN resolved; C = its high half (slot G+t of thread t is C's words tM ..),
// then the final subtraction (skipped when lazy); result in X
template <class W>
MPG_DI void cv_resolve_fma(const Grp<typename W::LS> &g, bool lazy) {
    constexpr int M = W::M;
    uint32_t in0[M + 2], fin[2][M];
    zero<M + 2>(in0);
    const uint32_t top = cv_resolve<W, M, PAT_SEQ>(g, in0, g.T(), PadMap<W::PAD>{}, fin);
    uint32_t c[2][M];
#pragma unroll
    for (int j = 0; j < M; ++j) { c[0][j] = fin[1][j]; c[1][j] = 0u; }
    if (lazy) sts<M>(g.X() + g.t * M, c[0]);
    else cv_cond_sub<W, M, PAT_ONE>(g, c, top, g.N(), g.X());
}

// X <- X * Y * R^-1 mod N, or X^2 * R^-1 mod N (Y then unused); Y holds q afterwards.
// On entry the operands are in shared memory behind a block barrier; on exit X holds the
// result behind a block barrier. lazy: no final subtraction (results < 2N when 4N <= R).
template <class W, int RED>
MPG_DI void swap_mont(const Views<W> &v, bool square, bool lazy) {
    const auto &gp = v.p;
    const auto &gl = v.l;
    // 1. T = X * Y or X^2 (slot sums in the product view, carries in the carry view)
    if (square) swp_sqr_slots<W>(gp, gp.X(), gp.T());
    else swp_mul_slots<W>(gp, gp.X(), gp.Y(), gp.T());
    bsync();
    uint32_t c_add, low_zero;
    cv_resolve_T<W>(gl, c_add, low_zero);
    bsync();
    // 2. q = T_lo * N' mod R
    swp_mullo_slots<W>(gp, gp.T(), gp.NI(), gp.Q());
    bsync();
    cv_resolve_q<W>(gl);
    bsync();
    if constexpr (RED == 0) {
        // 3. C = floor(T/R) + floor(qN/R) + c_add from the high half of qN (Thm. 2)
        swp_mulhi_slots<W>(gp, gp.Q(), gp.N(), gp.X(), gp.T());
        bsync();
        cv_resolve_hi<W>(gl, c_add, low_zero, lazy);
    } else {
        // 3. classical: T + q*N over all words, C = its high half
        (void)c_add;
        (void)low_zero;
        swp_fma_slots<W>(gp, gp.Q(), gp.N(), gp.T());
        bsync();
        cv_resolve_fma<W>(gl, lazy);
    }
    bsync();
}

// ------------------------------------------------------------------ kernels

template <class W>
constexpr int swap_blocks_per_sm() {
    constexpr long smem = (long)W::SMEM + 1024;
    constexpr long b = 233472L / smem;
    return b < 1 ? 1 : (int)b;
}

template <class W, int RED>
__global__ void __launch_bounds__(W::TPB, (swap_blocks_per_sm<W>())) k_mont_swap(KArgs A) {
    extern __shared__ uint4 smem4[];
    const Views<W> v = swap_views<W>(reinterpret_cast<uint32_t *>(smem4));
    using PS = typename W::PS;
    const Grp<PS> &g = v.p;
    const size_t k = swap_instance();
    const bool valid = k < A.batch;
    load_ctx<PS>(g, g.N(), A.N, A, k, valid);
    load_ctx<PS>(g, g.NI(), A.NI, A, k, valid);
    load_api<PS>(g, g.X(), A.a, A, k, valid);
    if (!A.square) load_api<PS>(g, g.Y(), A.b, A, k, valid);
    bsync();
    for (int r = 0; r <= (A.correct ? 1 : 0); ++r) {
        if (r) {
            load_ctx<PS>(g, g.Y(), A.K, A, k, valid);
            bsync();
        }
        swap_mont<W, RED>(v, r == 0 && A.square != 0, false);
    }
    uint32_t x[W::M];
    lds<W::M>(x, g.X() + g.t * W::M);
    gstore<W::M>(A.out, x, A.layout, k, valid, g.t * W::M, A.n, A.batch);
}

// Constant-time exponentiation (Alg. 7) in the role-swapped mapping: the same schedule as
// modexp_group, with table accesses and global loads in the product view.
// words between two instances' window tables in shared memory: 2^w entries of NP words, plus 4
// so that 32 instances' 16-byte accesses at one offset fall on distinct banks (as the records)
template <class W>
__host__ __device__ constexpr int tab_stride(int w) { return (1 << w) * W::NP + 4; }

template <class W>
constexpr size_t tab_smem(int w) { return W::SMEM + (size_t)32 * tab_stride<W>(w) * 4; }

template <class W, int RED, bool TAB = false>
MPG_DI void modexp_swap(const Views<W> &v, const KArgs &A, size_t k) {
    using PS = typename W::PS;
    constexpr int M = W::M;
    const Grp<PS> &g = v.p;
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
    // TAB: this instance's table in shared memory after the block's 32 records, entries of NP
    // words, instances tab_stride(w) words apart
    uint32_t *ts = nullptr;
    if constexpr (TAB) ts = v.p.sm - (size_t)(threadIdx.x & 31) * W::WORDS + 32 * W::WORDS +
                            (size_t)(threadIdx.x & 31) * tab_stride<W>(w);

    auto put = [&](int e, const uint32_t *src) {   // this thread's M words -> table entry e
        uint32_t x[M];
        lds<M>(x, src + g.t * M);
#ifdef MPG_DEBUG_BOUNDS
        if (valid && !dbg_ok(e >= 0 && e < E && kt < tb, DBG_TABLE, (unsigned long long)e * tb + kt)) return;
#endif
        if constexpr (TAB) {
            sts<M>(ts + e * W::NP + g.t * M, x);
            return;
        }
        if (!valid) return;
        if constexpr (M % 4 == 0) {
#pragma unroll
            for (int c = 0; c < M / 4; ++c)
                tab[tidx4<PS>(e, g.t * (M / 4) + c, kt, tb)] = make_uint4(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
        } else {
#pragma unroll
            for (int j = 0; j < M; ++j) {
                const int i = g.t * M + j;
                A.table[tidx4<PS>(e, i >> 2, kt, tb) * 4 + (i & 3)] = x[j];
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
        if constexpr (TAB) {
            lds<M>(x, ts + e * W::NP + g.t * M);
        } else if constexpr (M % 4 == 0) {
#pragma unroll
            for (int c = 0; c < M / 4; ++c) {
                uint4 q = make_uint4(0, 0, 0, 0);
                if (valid) q = tab[tidx4<PS>(e, g.t * (M / 4) + c, kt, tb)];
                x[4 * c] = q.x; x[4 * c + 1] = q.y; x[4 * c + 2] = q.z; x[4 * c + 3] = q.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < M; ++j) {
                const int i = g.t * M + j;
                x[j] = valid ? A.table[tidx4<PS>(e, i >> 2, kt, tb) * 4 + (i & 3)] : 0u;
            }
        }
    };

    load_ctx<PS>(g, g.N(), A.N, A, kc, valid);
    load_ctx<PS>(g, g.NI(), A.NI, A, kc, valid);
    const int nbuild = A.mode != 2 ? E - 1 : 0;
    const int windows = (A.ebits + w - 1) / w;
    const int nwin = A.mode != 1 ? windows * (w + 1) + 1 : 0;
    if (A.mode != 2) {
        load_api<PS>(g, g.X(), A.a, A, kt, valid);
        load_ctx<PS>(g, g.Y(), A.R2, A, kc, valid);
    } else {
        load_ctx<PS>(g, g.X(), A.R1, A, kc, valid);     // Y_acc = 1 in Montgomery form
    }
    bsync();
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
                bsync();
            } else if (s < w) {
                square = true;
            } else {   // masked scan of the whole table: every entry is read, one is kept
                const uint32_t bsel = window_bits(A, k, valid, (windows - 1 - i) * w, w);
                uint32_t acc[M];
                zero<M>(acc);
                // two entries per iteration: their loads are in flight together (measured best
                // of 1, 2, 4, 8: 2048-bit modexp 306.3k, 310.5k, 307.9k, 308.4k/s)
                constexpr int SCAN = 2;
                for (int e0 = 0; e0 < E; e0 += SCAN) {
                    uint32_t x[SCAN][M];
#pragma unroll
                    for (int r = 0; r < SCAN; ++r) {
                        if (e0 + r < E) fetch(e0 + r, x[r]);
                        else zero<M>(x[r]);
                    }
#pragma unroll
                    for (int r = 0; r < SCAN; ++r) {
                        const uint32_t m = mask_if_equal((uint32_t)(e0 + r), bsel);
#pragma unroll
                        for (int j = 0; j < M; ++j) acc[j] |= x[r][j] & m;
                    }
                }
                sts<M>(g.Y() + g.t * M, acc);
                bsync();
            }
        }
        swap_mont<W, RED>(v, square, A.lazy != 0);
        if (op < nbuild) {
            put(op + 1, g.X());
            if (op == 0) {                              // G[0] = R mod N
                load_ctx<PS>(g, g.Y(), A.R1, A, kc, valid);
                put(0, g.Y());
            }
            if (op + 1 < nbuild) {                      // next: G[op+2] = G[op+1] * G[1]
                uint32_t x[M];                          // (the product leaves q in Y)
                fetch(1, x);
                sts<M>(g.Y() + g.t * M, x);
            } else if (A.mode == 0) {
                load_ctx<PS>(g, g.X(), A.R1, A, kc, valid);   // Y_acc = 1 in Montgomery form
            }
            bsync();
        }
    }
    if (A.mode == 1) return;
    if (A.lazy) {   // X <= N here: one subtraction makes it canonical (carry view)
        cond_sub<typename W::LS>(v.l, v.l.X(), 0u, v.l.N(), v.l.X());
        bsync();
    }
    uint32_t x[M];
    lds<M>(x, g.X() + g.t * M);
    gstore<M>(A.out, x, A.layout, k, valid, g.t * M, A.n, A.batch);
}

template <class W, int RED, bool TAB = false>
__global__ void __launch_bounds__(W::TPB, (swap_blocks_per_sm<W>())) k_modexp_swap(KArgs A) {
    extern __shared__ uint4 smem4[];
    const Views<W> v = swap_views<W>(reinterpret_cast<uint32_t *>(smem4));
    const size_t k = swap_instance();
    const long long t0 = clock64();
    modexp_swap<W, RED, TAB>(v, A, k);
    if (A.cycles && v.p.t == 0 && k < A.batch) A.cycles[k] = (unsigned long long)(clock64() - t0);
}

// launchers: red 0 truncated, 1 classical; the word-serial reduction (red 2) passes a word
// between the threads of an instance at every step and keeps the lane-mapped kernels
template <class W, int KIND, class F>
static cudaError_t launch_swap(F kern, const KArgs &A, cudaStream_t st) {
    static std::atomic<unsigned long long> attr_done{0ull};
    const cudaError_t e = smem_attr_once(attr_done, kern, W::SMEM);
    if (e != cudaSuccess) return e;
    const size_t blocks = (A.batch + 31) / 32;
    kern<<<(unsigned)blocks, W::TPB, W::SMEM, st>>>(A);
    return cudaGetLastError();
}

template <class W, class Lane>
struct SwapImpl {
    static cudaError_t mont(const KArgs &A, cudaStream_t st) {
        if (A.red == 2) return Lane::mont(A, st);
        return A.red ? launch_swap<W, 1>(k_mont_swap<W, 1>, A, st) : launch_swap<W, 0>(k_mont_swap<W, 0>, A, st);
    }
    static cudaError_t modexp(const KArgs &A, cudaStream_t st) {
        if (A.red == 2) return Lane::modexp(A, st);
        if (A.tab_shared && A.mode == 0 && A.red == 0 && tab_fits(A.window)) return launch_tab(A, st);
        return A.red ? launch_swap<W, 3>(k_modexp_swap<W, 1>, A, st) : launch_swap<W, 2>(k_modexp_swap<W, 0>, A, st);
    }
    // the truncated exponentiation with its tables in shared memory fits one block on an SM
    static bool tab_fits(int w) {
        int dev = 0, optin = 0;
        if (w < 1 || w > 6 || cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            return false;
        return tab_smem<W>(w) <= (size_t)optin;
    }
    static cudaError_t launch_tab(const KArgs &A, cudaStream_t st) {
        static std::atomic<unsigned long long> attr_done{0ull};
        int dev = 0, optin = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess) e = smem_attr_once(attr_done, k_modexp_swap<W, 0, true>, (size_t)optin);
        if (e != cudaSuccess) return e;
        const size_t blocks = (A.batch + 31) / 32;
        k_modexp_swap<W, 0, true><<<(unsigned)blocks, W::TPB, tab_smem<W>(A.window), st>>>(A);
        return cudaGetLastError();
    }
    static int residency_tab(int w) {
        if (!tab_fits(w)) return 0;
        int dev = 0, optin = 0, blocks = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
            cudaFuncSetAttribute(k_modexp_swap<W, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_modexp_swap<W, 0, true>, W::TPB, tab_smem<W>(w)) !=
                cudaSuccess)
            return -1;
        return blocks * 32;
    }
    static int residency(int red) {
        if (red == 2) return Lane::residency(2);
        return red ? resident_instances(k_modexp_swap<W, 1>, W::TPB, W::SMEM, 32)
                   : resident_instances(k_modexp_swap<W, 0>, W::TPB, W::SMEM, 32);
    }
};

}  // namespace mpg

// a lane-mapped shape whose truncated and classical Montgomery kernels run role-swapped
#define MPG_DEFINE_SHAPE_SWAP(G, M, TPB)                                                     \
    namespace mpg {                                                                          \
    ShapeOps shape_ops_##G##_##M() {                                                         \
        using Lane = ShapeImpl<Shape<G, M>, TPB>;                                            \
        ShapeOps o = Lane::ops();                                                            \
        o.mont = &SwapImpl<Swap<G, M>, Lane>::mont;                                          \
        o.modexp = &SwapImpl<Swap<G, M>, Lane>::modexp;                                      \
        o.residency = &SwapImpl<Swap<G, M>, Lane>::residency;                                \
        o.residency_tab = &SwapImpl<Swap<G, M>, Lane>::residency_tab;                        \
        return o;                                                                            \
    }                                                                                        \
    }

#define MPG_DEFINE_SHAPE_KARA_SWAP(G, M, TPB, MH, TPBK)                                      \
    namespace mpg {                                                                          \
    ShapeOps shape_ops_##G##_##M() {                                                         \
        using Lane = ShapeImpl<Shape<G, M>, TPB>;                                            \
        ShapeOps o = Lane::ops();                                                            \
        o.kara = &launch_kara<Shape<G, M>, Shape<G, MH>, TPBK>;                              \
        o.mont = &SwapImpl<Swap<G, M>, Lane>::mont;                                          \
        o.modexp = &SwapImpl<Swap<G, M>, Lane>::modexp;                                      \
        o.residency = &SwapImpl<Swap<G, M>, Lane>::residency;                                \
        o.residency_tab = &SwapImpl<Swap<G, M>, Lane>::residency_tab;                        \
        return o;                                                                            \
    }                                                                                        \
    }
