// Role-swapped batched products: schoolbook (Sec. 2.1, Alg. 1-2) and one level of Karatsuba
// (Sec. 3) under the two thread mappings of mp_swap.cuh (product view: warp t plays thread t of
// 32 instances; carry view: G consecutive lanes per instance).
//
// Karatsuba, operands of 2h words (h = G*M), A = a_l + W^h a_h, B = b_l + W^h b_h:
//   D0 = a_l b_l,  D2 = a_h b_h,  D1' = (a_l + a_h)(b_l + b_h)
//   A*B = D0 + W^h (D1' - D0 - D2) + W^2h D2.
// s_a = a_l + a_h is formed as h words plus a carry bit c_a, so
//   D1' = s_a s_b + W^h (c_a s_b + c_b s_a) + W^2h c_a c_b.
// The three half products run as role-swapped schoolbook products of G roles x M words; D0 and
// D2 are resolved and stored over their operands, and the recombination is folded into the slot
// sums of the last one. With R = A*B, D0 = D0_lo + W^h D0_hi, D2 = D2_lo + W^h D2_hi and
// ~D = W^(2h+1) - 1 - D (complement over 2h+1 words):
//   Y = D0_hi + (D1' - D0 - D2) + W^h D2_lo < W^(2h+1),   R = D0_lo + W^h Y + W^3h D2_hi
//   Z = D1' + ~D0 + ~D2 + 2 + D0_hi + W^h D2_lo = Y + 2 W^(2h+1),  so Y = Z mod W^(2h+1).
// Every term of Z is non-negative and lands on the columns of one slot of D1 owned by the role
// that computes that slot, which adds it before the slot is stored; one resolution gives Y, and
// the carry out of Y into D2_hi is resolved across the group with the usual lookahead.
#pragma once
#include "mp_kara.cuh"
#include "mp_swap.cuh"

namespace mpg {

// Record of a schoolbook product: X, Y (NP words each), T (2NP, padded), spills
template <int G_, int M_>
struct SwapMul {
    using PS = Shape<G_, M_, true>;
    using LS = Shape<G_, M_, false>;
    static constexpr int G = G_, M = M_, NP = G_ * M_;
    static constexpr int TPB = 32 * G_;
    static_assert(32 % G_ == 0, "the G threads of an instance share a warp in the carry view");
    static constexpr bool PAD = (M_ % 8 == 0);
    static constexpr int OFF_X = 0, OFF_Y = NP;
    static constexpr int OFF_T = 2 * NP;
    static constexpr int OFF_P = (OFF_T + pad_size(2 * NP, PAD) + 3) & ~3;
    static constexpr int SPILL_TOP = (pad_size(2 * G * M, PAD) + 3) & ~3;
    static constexpr int WORDS_RAW = OFF_P + SPILL_TOP + 2 * G;
    static constexpr int WORDS = ((WORDS_RAW + 3) / 8) * 8 + 4;   // 4 (mod 8): see Swap
    static constexpr size_t SMEM = (size_t)32 * WORDS * 4;
    // registers a thread needs without spilling (the M-word blocks' accumulator and operands)
    static constexpr int MIN_REGS = M_ <= 4 ? 64 : M_ <= 8 ? 80 : 128;
};

// Record of a one-level Karatsuba product whose half products run on G roles x M words
// (h = G*M words per half, operands of 2h words): [a_l | b_l | a_h | b_h], later [D0 | D2];
// s_a | s_b; T (2h, padded); spills; c_a, c_b
template <int G_, int M_>
struct SwapKara {
    using PS = Shape<G_, M_, true>;
    using LS = Shape<G_, M_, false>;
    static constexpr int G = G_, M = M_, NP = G_ * M_, h = NP;
    static constexpr int TPB = 32 * G_;
    static_assert(32 % G_ == 0, "the G threads of an instance share a warp in the carry view");
    static constexpr bool PAD = (M_ % 8 == 0);
    static constexpr int OFF_D = 0;
    static constexpr int OFF_S = 4 * h;
    static constexpr int OFF_T = 6 * h;
    static constexpr int OFF_P = (OFF_T + pad_size(2 * h, PAD) + 3) & ~3;
    static constexpr int SPILL_TOP = (pad_size(2 * G * M, PAD) + 3) & ~3;
    static constexpr int OFF_C = OFF_P + SPILL_TOP + 2 * G;
    static constexpr int WORDS_RAW = OFF_C + 2;
    static constexpr int WORDS = ((WORDS_RAW + 3) / 8) * 8 + 4;
    static constexpr size_t SMEM = (size_t)32 * WORDS * 4;
    static constexpr int MIN_REGS = M_ <= 4 ? 64 : M_ <= 6 ? 80 : 128;
};

// blocks per SM: as many as shared memory allows, but no fewer than MIN_REGS registers a thread
template <class W>
constexpr int prod_blocks_per_sm() {
    constexpr int by_smem = swap_blocks_per_sm<W>();
    constexpr int by_regs = 65536 / (W::TPB * W::MIN_REGS);
    constexpr int b = by_smem < by_regs ? by_smem : by_regs;
    return b < 1 ? 1 : b;
}

// instance of the carry view in the launch
template <class W>
MPG_DI size_t swap_instance_cv() {
    return (size_t)blockIdx.x * 32 + (threadIdx.x >> 5) * (32 / W::G) + (threadIdx.x & 31) / W::G;
}

// resolve the slot sums in T (and the spills) into this lane's two slots (t and G+t) of
// B-word words; returns the low word above the last slot
template <class W, int B>
MPG_DI uint32_t swk_resolve(const Grp<typename W::LS> &g, const uint32_t *T, uint32_t (&fin)[2][B]) {
    uint32_t in0[B + 2];
    zero<B + 2>(in0);
    return cv_resolve<W, B, PAT_SEQ>(g, in0, T, PadMap<W::PAD>{}, fin);
}

// ------------------------------------------------------------------ schoolbook

template <class W>
__global__ void __launch_bounds__(W::TPB, (prod_blocks_per_sm<W>())) k_mul_swap(KArgs A) {
    extern __shared__ uint4 smem4[];
    const Views<W> v = swap_views<W>(reinterpret_cast<uint32_t *>(smem4));
    using PS = typename W::PS;
    constexpr int M = W::M, G = W::G;
    const Grp<PS> &g = v.p;
    {
        const size_t k = swap_instance();
        const bool valid = k < A.batch;
        load_api<PS>(g, g.sm + W::OFF_X, A.a, A, k, valid);
        if (!A.square) load_api<PS>(g, g.sm + W::OFF_Y, A.b, A, k, valid);
    }
    bsync();
    if (A.square) swp_sqr_slots<W>(g, g.sm + W::OFF_X, g.sm + W::OFF_T);
    else swp_mul_slots<W>(g, g.sm + W::OFF_X, g.sm + W::OFF_Y, g.sm + W::OFF_T);
    bsync();
    const auto &gl = v.l;
    uint32_t fin[2][M];
    swk_resolve<W, M>(gl, gl.sm + W::OFF_T, fin);   // the product is below W^(2NP): nothing above
    const size_t k = swap_instance_cv<W>();
    const bool valid = k < A.batch;
    gstore<M>(A.out, fin[0], A.layout, k, valid, gl.t * M, 2 * A.n, A.batch);
    gstore<M>(A.out, fin[1], A.layout, k, valid, (G + gl.t) * M, 2 * A.n, A.batch);
}

// ------------------------------------------------------------------ one level of Karatsuba

// z[0 .. M+2) += x[0 .. M)
template <int M>
MPG_DI void acc_add(uint32_t (&z)[M + 2], const uint32_t (&x)[M]) {
    add_cc(z[0], x[0]);
#pragma unroll
    for (int j = 1; j < M; ++j) addc_cc(z[j], x[j]);
    addc_cc(z[M], 0u);
    addc(z[M + 1], 0u);
}

// Slot sums of Z (see the top of the file) in the product view: the slots of D1' = s_a s_b
// (or s_a^2) with the other terms of Z added by the role that owns their columns.
//   slot t   (Z columns tM ..):      ~D0_t + ~D2_t + D0_{G+t}          (+2 for t = 0)
//   slot G+t (Z columns h + tM ..):  ~D0_{G+t} + ~D2_{G+t} + D2_t + c_a s_b,t + c_b s_a,t
//                                    (t = G-1: + 2(W-1) + c_a c_b at column 2h, local word M)
// D0 and D2 are the resolved half products at D and D + 2h.
template <class W, bool SQR>
MPG_DI void swk_z_slots(const Grp<typename W::PS> &g, const uint32_t *SA, const uint32_t *SB, const uint32_t *D,
                        uint32_t ca, uint32_t cb, uint32_t *T) {
    constexpr int G = W::G, M = W::M, h = W::h, U = run_group<M>();
    const int t = g.t;
    const bool even = (t & 1) == 0;
    Acc3<M> a;
    uint32_t top[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int s = k ? G + t : t;
        acc3_zero<M>(a);
        uint32_t V[2 * M + 2];
        if constexpr (SQR) {
            const int nA = (t + 1) >> 1, nB = ((G - t + 1) >> 1) - 1;
            if (k == 0) mac_run<M, U>(a, SA, SA, nA, [&](int j, int &u, int &v) { u = j; v = t - j; });
            else mac_run<M, U>(a, SA, SA, nB, [&](int j, int &u, int &v) { u = t + 1 + j; v = G - 1 - j; });
            uint32_t x[M];
            if (even) {
                lds<M>(x, SA + (s >> 1) * M);
                acc3_tri<M>(a, x);
            } else {
                zero<M>(x);
            }
            acc3_value<M>(V, a);
            double_add_diag<M>(V, x);
        } else {
            if (k == 0) mac_run<M, U>(a, SA, SB, t + 1, [&](int j, int &u, int &v) { u = j; v = t - j; });
            else mac_run<M, U>(a, SA, SB, G - 1 - t, [&](int j, int &u, int &v) { u = t + 1 + j; v = G - 1 - j; });
            acc3_value<M>(V, a);
        }
        uint32_t x[M], z[M + 2];
        lds<M>(x, D + s * M);            // ~D0 segment s
#pragma unroll
        for (int j = 0; j < M; ++j) z[j] = ~x[j];
        z[M] = 0u;
        z[M + 1] = 0u;
        lds<M>(x, D + 2 * h + s * M);    // ~D2 segment s
#pragma unroll
        for (int j = 0; j < M; ++j) x[j] = ~x[j];
        acc_add<M>(z, x);
        if (k == 0) {
            lds<M>(x, D + (G + t) * M);  // D0_hi segment t
            acc_add<M>(z, x);
            if (t == 0) {
                zero<M>(x);
                x[0] = 2u;
                acc_add<M>(z, x);
            }
        } else {
            lds<M>(x, D + 2 * h + t * M);   // D2_lo segment t
            acc_add<M>(z, x);
            const uint32_t ma = 0u - ca, mb = 0u - cb;
            lds<M>(x, SB + t * M);
#pragma unroll
            for (int j = 0; j < M; ++j) x[j] &= ma;
            acc_add<M>(z, x);
            lds<M>(x, SA + t * M);
#pragma unroll
            for (int j = 0; j < M; ++j) x[j] &= mb;
            acc_add<M>(z, x);
        }
        add_cc(V[0], z[0]);
#pragma unroll
        for (int j = 1; j < M + 2; ++j) addc_cc(V[j], z[j]);
#pragma unroll
        for (int j = M + 2; j < 2 * M + 1; ++j) addc_cc(V[j], 0u);
        addc(V[2 * M + 1], 0u);
        if (k == 1 && t == G - 1) {   // column 2h: 2(W-1) + c_a c_b = W + (W - 2 + c_a c_b)
            add_cc(V[M], 0xfffffffeu + (ca & cb));
            addc_cc(V[M + 1], 1u);
#pragma unroll
            for (int j = M + 2; j < 2 * M + 1; ++j) addc_cc(V[j], 0u);
            addc(V[2 * M + 1], 0u);
        }
        top[k] = store_lohi<M>(V, T + pad32<W::PAD>(s * M), swp_hi<W, M>(g, s));
    }
    store_tops<W>(g, top[0], top[1]);
}

template <class W>
__global__ void __launch_bounds__(W::TPB, (prod_blocks_per_sm<W>())) k_kara_swap(KArgs A) {
    extern __shared__ uint4 smem4[];
    const Views<W> v = swap_views<W>(reinterpret_cast<uint32_t *>(smem4));
    using PS = typename W::PS;
    constexpr int M = W::M, G = W::G, h = W::h;
    const Grp<PS> &gp = v.p;
    const auto &gl = v.l;
    const bool sqr = A.square != 0;
    {   // a -> [a_l | . | a_h | .], b -> [. | b_l | . | b_h]; warp t loads words 2tM .. 2tM+2M
        const size_t k = swap_instance();
        const bool valid = k < A.batch;
        const int w0 = 2 * gp.t * M;
        const int hi = w0 >= h ? h : 0;
        uint32_t x[2 * M];
        gload<2 * M>(x, A.a, A.layout, k, valid, w0, A.n, A.batch);
        sts<2 * M>(gp.sm + W::OFF_D + w0 + hi, x);
        if (!sqr) {
            gload<2 * M>(x, A.b, A.layout, k, valid, w0, A.n, A.batch);
            sts<2 * M>(gp.sm + W::OFF_D + h + w0 + hi, x);
        }
    }
    bsync();
    // carry view: s_a = a_l + a_h, s_b = b_l + b_h (no barrier before D0: disjoint words)
    {
        uint32_t *D = gl.sm + W::OFF_D, *S = gl.sm + W::OFF_S;
        const uint32_t ca = gadd<typename W::LS, M>(gl, S, D, [&](int i) { return D[2 * h + i]; }, 0u);
        uint32_t cb = ca;
        if (!sqr) cb = gadd<typename W::LS, M>(gl, S + h, D + h, [&](int i) { return D[3 * h + i]; }, 0u);
        if (gl.t == 0) {
            gl.sm[W::OFF_C] = ca;
            gl.sm[W::OFF_C + 1] = cb;
        }
    }
    uint32_t *Dp = gp.sm + W::OFF_D, *Tp = gp.sm + W::OFF_T;
    uint32_t *Dl = gl.sm + W::OFF_D, *Tl = gl.sm + W::OFF_T;
    uint32_t fin[2][M];
    // D0 = a_l b_l over [a_l | b_l]
    if (sqr) swp_sqr_slots<W>(gp, Dp, Tp);
    else swp_mul_slots<W>(gp, Dp, Dp + h, Tp);
    bsync();
    swk_resolve<W, M>(gl, Tl, fin);
    sts<M>(Dl + gl.t * M, fin[0]);
    sts<M>(Dl + (G + gl.t) * M, fin[1]);
    bsync();
    // D2 = a_h b_h over [a_h | b_h]
    if (sqr) swp_sqr_slots<W>(gp, Dp + 2 * h, Tp);
    else swp_mul_slots<W>(gp, Dp + 2 * h, Dp + 3 * h, Tp);
    bsync();
    swk_resolve<W, M>(gl, Tl, fin);
    sts<M>(Dl + 2 * h + gl.t * M, fin[0]);
    sts<M>(Dl + 2 * h + (G + gl.t) * M, fin[1]);
    bsync();
    // Z = D1' + ~D0 + ~D2 + 2 + D0_hi + W^h D2_lo
    {
        const uint32_t ca = gp.sm[W::OFF_C], cb = gp.sm[W::OFF_C + 1];
        const uint32_t *S = gp.sm + W::OFF_S;
        if (sqr) swk_z_slots<W, true>(gp, S, S, Dp, ca, ca, Tp);
        else swk_z_slots<W, false>(gp, S, S + h, Dp, ca, cb, Tp);
    }
    bsync();
    // carry view: Y = Z mod W^(2h+1) (R words h .. 3h and the word above), then R's top quarter
    // D2_hi + Y_2h with the carries resolved across the group
    const uint32_t top = swk_resolve<W, M>(gl, Tl, fin);
    uint32_t lo[M], q[M];
    lds<M>(lo, Dl + gl.t * M);                     // R segment t = D0 segment t
    lds<M>(q, Dl + 2 * h + (G + gl.t) * M);        // D2_hi segment t
    const uint32_t gen = add_word<M>(q, gl.t == 0 ? top : 0u);
    uint32_t pall = q[0];
#pragma unroll
    for (int j = 1; j < M; ++j) pall &= q[j];
    const uint64_t Gm = gl.gbits(gen != 0u), Pm = gl.gbits(pall == 0xffffffffu);
    const uint64_t cin = (Pm + (Gm << 1)) ^ Pm;
    add_word<M>(q, (uint32_t)(cin >> gl.t) & 1u);
    const size_t k = swap_instance_cv<W>();
    const bool valid = k < A.batch;
    const int nw = 2 * A.n;
    gstore<M>(A.out, lo, A.layout, k, valid, gl.t * M, nw, A.batch);
    gstore<M>(A.out, fin[0], A.layout, k, valid, h + gl.t * M, nw, A.batch);
    gstore<M>(A.out, fin[1], A.layout, k, valid, 2 * h + gl.t * M, nw, A.batch);
    gstore<M>(A.out, q, A.layout, k, valid, 3 * h + gl.t * M, nw, A.batch);
}

template <class W, class F>
static cudaError_t launch_swap_prod(F kern, std::atomic<unsigned long long> &attr_done, const KArgs &A,
                                    cudaStream_t st) {
    const cudaError_t e = smem_attr_once(attr_done, kern, W::SMEM);
    if (e != cudaSuccess) return e;
    const size_t blocks = (A.batch + 31) / 32;
    kern<<<(unsigned)blocks, W::TPB, W::SMEM, st>>>(A);
    return cudaGetLastError();
}

template <class W>
static cudaError_t launch_mul_swap(const KArgs &A, cudaStream_t st) {
    static std::atomic<unsigned long long> attr_done{0ull};
    return launch_swap_prod<W>(k_mul_swap<W>, attr_done, A, st);
}

template <class W>
static cudaError_t launch_kara_swap(const KArgs &A, cudaStream_t st) {
    static std::atomic<unsigned long long> attr_done{0ull};
    return launch_swap_prod<W>(k_kara_swap<W>, attr_done, A, st);
}

}  // namespace mpg

// Shape (G, M) with role-swapped Montgomery kernels, role-swapped schoolbook products on GP roles
// x MP words and a role-swapped one-level Karatsuba product over half products of GK roles x MK
// words
#define MPG_DEFINE_SHAPE_SWAP_ALL(G, M, TPB, GP, MP, GK, MK)                                         \
    namespace mpg {                                                                          \
    ShapeOps shape_ops_##G##_##M() {                                                         \
        using Lane = ShapeImpl<Shape<G, M>, TPB>;                                            \
        ShapeOps o = Lane::ops();                                                            \
        o.mul = &launch_mul_swap<SwapMul<GP, MP>>;                                           \
        o.kara = &launch_kara_swap<SwapKara<GK, MK>>;                                        \
        o.mont = &SwapImpl<Swap<G, M>, Lane>::mont;                                          \
        o.modexp = &SwapImpl<Swap<G, M>, Lane>::modexp;                                      \
        o.residency = &SwapImpl<Swap<G, M>, Lane>::residency;                                \
        o.residency_tab = &SwapImpl<Swap<G, M>, Lane>::residency_tab;                        \
        return o;                                                                            \
    }                                                                                        \
    }

// Shape (G, M) with lane-mapped Montgomery kernels and role-swapped products
#define MPG_DEFINE_SHAPE_PROD_SWAP(G, M, TPB, GP, MP, GK, MK)                                        \
    namespace mpg {                                                                          \
    ShapeOps shape_ops_##G##_##M() {                                                         \
        ShapeOps o = ShapeImpl<Shape<G, M>, TPB>::ops();                                     \
        o.mul = &launch_mul_swap<SwapMul<GP, MP>>;                                           \
        o.kara = &launch_kara_swap<SwapKara<GK, MK>>;                                        \
        return o;                                                                            \
    }                                                                                        \
    }
