// 32-bit limb primitives: IMAD / IMAD.HI carry chains written as inline PTX.
//
// The paper's primitive is the 52-bit fused multiply-add VPMADD52 (lo and hi
// halves, Sec. 2). Its GPU counterpart is the 32x32-bit multiply-add in two
// halves, mad.lo.cc.u32 / madc.hi.cc.u32, chained through the carry flag.
// Every function here runs the same instruction sequence for every input value.
#pragma once
#include <cstdint>
#include "mp_debug.cuh"

namespace mpg {

#define MPG_DI __device__ __forceinline__

MPG_DI void add_cc(uint32_t &a, uint32_t b) { asm volatile("add.cc.u32 %0, %0, %1;" : "+r"(a) : "r"(b)); }
MPG_DI void addc_cc(uint32_t &a, uint32_t b) { asm volatile("addc.cc.u32 %0, %0, %1;" : "+r"(a) : "r"(b)); }
MPG_DI void addc(uint32_t &a, uint32_t b) { asm volatile("addc.u32 %0, %0, %1;" : "+r"(a) : "r"(b)); }
MPG_DI uint32_t addc_get(void) { uint32_t r; asm volatile("addc.u32 %0, 0, 0;" : "=r"(r)); return r; }
MPG_DI void sub_cc(uint32_t &a, uint32_t b) { asm volatile("sub.cc.u32 %0, %0, %1;" : "+r"(a) : "r"(b)); }
MPG_DI void subc_cc(uint32_t &a, uint32_t b) { asm volatile("subc.cc.u32 %0, %0, %1;" : "+r"(a) : "r"(b)); }
// borrow flag after a sub chain, as 0/1
MPG_DI uint32_t subc_borrow(void) { uint32_t r; asm volatile("subc.u32 %0, 0, 0;" : "=r"(r)); return r & 1u; }

MPG_DI void mad_lo_cc(uint32_t &acc, uint32_t a, uint32_t b) {
    asm volatile("mad.lo.cc.u32 %0, %1, %2, %0;" : "+r"(acc) : "r"(a), "r"(b));
}
MPG_DI void madc_lo_cc(uint32_t &acc, uint32_t a, uint32_t b) {
    asm volatile("madc.lo.cc.u32 %0, %1, %2, %0;" : "+r"(acc) : "r"(a), "r"(b));
}
MPG_DI void mad_hi_cc(uint32_t &acc, uint32_t a, uint32_t b) {
    asm volatile("mad.hi.cc.u32 %0, %1, %2, %0;" : "+r"(acc) : "r"(a), "r"(b));
}
MPG_DI void madc_hi_cc(uint32_t &acc, uint32_t a, uint32_t b) {
    asm volatile("madc.hi.cc.u32 %0, %1, %2, %0;" : "+r"(acc) : "r"(a), "r"(b));
}

// P[0..2B) = x[0..B) * y[0..B): one B x B block of partial products (operand
// scanning). Row i adds x_i*y into P[i..i+B] with two carry chains: the
// "even" chain takes lo/hi of x_i*y_j for even j (lo at i+j, hi at i+j+1: the
// positions of one chain never collide), the "odd" chain the odd j. After
// row i the partial sum is below W^(i+B+1), so neither chain can carry out
// of position i+B: 2B IMAD plus one or two ADDC per row.
template <int B>
MPG_DI void block_mul(uint32_t (&P)[2 * B], const uint32_t (&x)[B], const uint32_t (&y)[B]) {
#pragma unroll
    for (int j = 0; j < 2 * B; ++j) P[j] = 0;
#pragma unroll
    for (int i = 0; i < B; ++i) {
        // even chain
        mad_lo_cc(P[i], x[i], y[0]);
        madc_hi_cc(P[i + 1], x[i], y[0]);
#pragma unroll
        for (int j = 2; j < B; j += 2) {
            madc_lo_cc(P[i + j], x[i], y[j]);
            madc_hi_cc(P[i + j + 1], x[i], y[j]);
        }
        {
            constexpr int last_even = ((B - 1) / 2) * 2;    // largest even j < B
#pragma unroll
            for (int p = last_even + 2; p <= B; ++p) addc_cc(P[i + p], 0u);
        }
        // odd chain
        if constexpr (B > 1) {
            mad_lo_cc(P[i + 1], x[i], y[1]);
            madc_hi_cc(P[i + 2], x[i], y[1]);
#pragma unroll
            for (int j = 3; j < B; j += 2) {
                madc_lo_cc(P[i + j], x[i], y[j]);
                madc_hi_cc(P[i + j + 1], x[i], y[j]);
            }
            constexpr int last_odd = ((B - 2) / 2) * 2 + 1;  // largest odd j < B
#pragma unroll
            for (int p = last_odd + 2; p <= B; ++p) addc_cc(P[i + p], 0u);
        }
    }
}

// P = x^2 (2B words) from the B(B-1)/2 cross products x_i x_j (i < j), doubled, plus the B
// squares x_i^2 at column 2i (Alg. 2's split, on one block).
template <int B>
MPG_DI void block_sqr(uint32_t (&P)[2 * B], const uint32_t (&x)[B]) {
#pragma unroll
    for (int j = 0; j < 2 * B; ++j) P[j] = 0;
#pragma unroll
    for (int i = 0; i + 1 < B; ++i) {
        // two chains per row (j - i odd, j - i even): their (lo, hi) pairs never share a column
#pragma unroll
        for (int par = 1; par <= 2; ++par) {
            if (i + par < B) {
#pragma unroll
                for (int j = i + par; j < B; j += 2) {
                    if (j == i + par) mad_lo_cc(P[i + j], x[i], x[j]);
                    else madc_lo_cc(P[i + j], x[i], x[j]);
                    madc_hi_cc(P[i + j + 1], x[i], x[j]);
                }
                const int jl = i + par + 2 * ((B - 1 - (i + par)) / 2);   // last j of the chain
#pragma unroll
                for (int p = i + jl + 2; p <= i + B; ++p) addc_cc(P[p], 0u);
            }
        }
    }
    // double: the cross sum is below W^(2B) / 2
#pragma unroll
    for (int k = 2 * B - 1; k > 0; --k) P[k] = __funnelshift_l(P[k - 1], P[k], 1);
    P[0] <<= 1;
    mad_lo_cc(P[0], x[0], x[0]);
    madc_hi_cc(P[1], x[0], x[0]);
#pragma unroll
    for (int i = 1; i < B; ++i) {
        madc_lo_cc(P[2 * i], x[i], x[i]);
        madc_hi_cc(P[2 * i + 1], x[i], x[i]);
    }
}

// V[0..2B+2) += P[0..2B)
template <int B>
MPG_DI void acc_add(uint32_t (&V)[2 * B + 2], const uint32_t (&P)[2 * B]) {
    add_cc(V[0], P[0]);
#pragma unroll
    for (int j = 1; j < 2 * B; ++j) addc_cc(V[j], P[j]);
    addc_cc(V[2 * B], 0u);
    addc(V[2 * B + 1], 0u);
}

// a[0..K) += b[0..K) with carry out (0/1)
template <int K>
MPG_DI uint32_t add_n(uint32_t (&a)[K], const uint32_t (&b)[K]) {
    add_cc(a[0], b[0]);
#pragma unroll
    for (int j = 1; j < K; ++j) addc_cc(a[j], b[j]);
    return addc_get();
}

// a[0..K) -= b[0..K), returns borrow (0/1)
template <int K>
MPG_DI uint32_t sub_n(uint32_t (&a)[K], const uint32_t (&b)[K]) {
    sub_cc(a[0], b[0]);
#pragma unroll
    for (int j = 1; j < K; ++j) subc_cc(a[j], b[j]);
    return subc_borrow();
}

// a[0..K) += c (c < 2^32) with carry out
template <int K>
MPG_DI uint32_t add_word(uint32_t (&a)[K], uint32_t c) {
    add_cc(a[0], c);
#pragma unroll
    for (int j = 1; j < K; ++j) addc_cc(a[j], 0u);
    return addc_get();
}

// a[0..K) -= c with borrow out
template <int K>
MPG_DI uint32_t sub_word(uint32_t (&a)[K], uint32_t c) {
    sub_cc(a[0], c);
#pragma unroll
    for (int j = 1; j < K; ++j) subc_cc(a[j], 0u);
    return subc_borrow();
}

// ------------------------------------------------------------------ split-column accumulator
//
// A chain of lo/hi pairs mad.lo.cc(c) / madc.hi.cc(c+1) adds one 64-bit partial product to
// the register pair (c, c+1); the multiply pipe executes it as one wide multiply-add, which
// reads and writes an aligned 64-bit register pair. In an operand-scanning row x_i * y the
// pairs start at columns i + j, so the chain over even j starts at columns of the parity of i
// and the chain over odd j at the other parity: with one array per block, the words that one
// row pairs as (c, c+1) the next row pairs as (c-1, c) and (c+1, c+2), and the compiler moves
// words around to assemble aligned pairs (measured: 16 extra multiply-pipe instructions and
// about 40 extra ALU instructions per 8 x 8 block, on top of the 64 wide multiply-adds).
// Acc3 keeps pairs that start at even columns in E and pairs that start at odd columns in O
// (shifted by one word), so every pair of every row lands on an aligned pair of one of them;
// the carry out of each row chain goes to a small counter word in K instead of rippling up.
//   value = sum_c E[c] W^c + sum_k O[k] W^(k+1) + sum_k K[k] W^(B+k)
// Each 64-bit step of a chain adds a pair, a product and a carry: below 2^65, so the carry out
// of every step, and of the chain, is 0 or 1; no word of E or O overflows and K[k] counts at
// most 2 per block product.
template <int B>
struct Acc3 {
    static_assert(B >= 2, "split accumulator: blocks of two words or more");
    uint32_t E[2 * B];       // columns 0 .. 2B-1
    uint32_t O[2 * B - 2];   // columns 1 .. 2B-2
    uint32_t K[B + 1];       // columns B .. 2B (chain carries)
};

template <int B>
MPG_DI void acc3_zero(Acc3<B> &a) {
#pragma unroll
    for (int j = 0; j < 2 * B; ++j) a.E[j] = 0u;
#pragma unroll
    for (int j = 0; j < 2 * B - 2; ++j) a.O[j] = 0u;
#pragma unroll
    for (int j = 0; j < B + 1; ++j) a.K[j] = 0u;
}

// one chain of NP pairs x * y[J0], x * y[J0+2], ... into the words D[D0], D[D0+1], ... (D0
// even), its carry out added to *k
template <int B, int LEN, int J0, int D0, int NP>
MPG_DI void acc3_chain(uint32_t (&D)[LEN], uint32_t &k, uint32_t x, const uint32_t (&y)[B]) {
    static_assert(D0 % 2 == 0 && D0 + 2 * NP <= LEN && J0 + 2 * (NP - 1) < B, "chain out of range");
    mad_lo_cc(D[D0], x, y[J0]);
    madc_hi_cc(D[D0 + 1], x, y[J0]);
#pragma unroll
    for (int p = 1; p < NP; ++p) {
        madc_lo_cc(D[D0 + 2 * p], x, y[J0 + 2 * p]);
        madc_hi_cc(D[D0 + 2 * p + 1], x, y[J0 + 2 * p]);
    }
    addc(k, 0u);
}

// row i: a += x_i * y * W^i as two chains, over even j and over odd j. The pairs of the
// chain over j = J0, J0+2, .. start at columns I+J0, I+J0+2, ...: in E (index = column) when
// that column is even, in O (index = column - 1) when it is odd. A chain whose last j is L
// carries into column I+L+2, i.e. K[I+L+2-B].
template <int B, int I>
MPG_DI void acc3_row(Acc3<B> &a, uint32_t xi, const uint32_t (&y)[B]) {
    constexpr int L0 = (B - 1) & ~1;    // last even j
    constexpr int L1 = (B - 2) | 1;     // last odd j
    constexpr int N0 = L0 / 2 + 1, N1 = (L1 + 1) / 2;
    if constexpr (I % 2 == 0) {
        acc3_chain<B, 2 * B, 0, I, N0>(a.E, a.K[I + L0 + 2 - B], xi, y);
        acc3_chain<B, 2 * B - 2, 1, I, N1>(a.O, a.K[I + L1 + 2 - B], xi, y);
    } else {
        acc3_chain<B, 2 * B - 2, 0, I - 1, N0>(a.O, a.K[I + L0 + 2 - B], xi, y);
        acc3_chain<B, 2 * B, 1, I + 1, N1>(a.E, a.K[I + L1 + 2 - B], xi, y);
    }
}

template <int B, int I = 0>
MPG_DI void acc3_rows(Acc3<B> &a, const uint32_t (&x)[B], const uint32_t (&y)[B]) {
    if constexpr (I < B) {
        acc3_row<B, I>(a, x[I], y);
        acc3_rows<B, I + 1>(a, x, y);
    }
}

// a += x * y (B x B words)
template <int B>
MPG_DI void acc3_mac(Acc3<B> &a, const uint32_t (&x)[B], const uint32_t (&y)[B]) {
    acc3_rows<B>(a, x, y);
}

// the cross terms of x^2: a += sum over i < j of x_i x_j W^(i+j) (row i: the chains over
// j = i+1, i+3, ... and j = i+2, i+4, ..., each pair in E or O by the parity of its column)
template <int B, int I, int J0>
MPG_DI void acc3_tri_chain(Acc3<B> &a, const uint32_t (&x)[B]) {
    if constexpr (J0 < B) {
        constexpr int NP = (B - J0 + 1) / 2;            // pairs j = J0, J0+2, ... < B
        constexpr int LAST = J0 + 2 * (NP - 1);
        constexpr int C0 = I + J0;                      // column of the first pair
        constexpr int KI = I + LAST + 2 - B;            // carry column I+LAST+2 in K
        static_assert(KI >= 0 && KI <= B, "carry column of a triangle chain");
        if constexpr (C0 % 2 == 0) acc3_chain<B, 2 * B, J0, C0, NP>(a.E, a.K[KI], x[I], x);
        else acc3_chain<B, 2 * B - 2, J0, C0 - 1, NP>(a.O, a.K[KI], x[I], x);
    }
}

template <int B, int I = 0>
MPG_DI void acc3_tri(Acc3<B> &a, const uint32_t (&x)[B]) {
    if constexpr (I + 1 < B) {
        acc3_tri_chain<B, I, I + 1>(a, x);
        acc3_tri_chain<B, I, I + 2>(a, x);
        acc3_tri<B, I + 1>(a, x);
    }
}

// V[0 .. 2B+2) = value of a
template <int B>
MPG_DI void acc3_value(uint32_t (&V)[2 * B + 2], const Acc3<B> &a) {
    V[0] = a.E[0];
#pragma unroll
    for (int j = 1; j < 2 * B; ++j) V[j] = a.E[j];
    V[2 * B] = 0u;
    V[2 * B + 1] = 0u;
    add_cc(V[1], a.O[0]);
#pragma unroll
    for (int j = 1; j < 2 * B - 2; ++j) addc_cc(V[1 + j], a.O[j]);
    addc_cc(V[2 * B - 1], 0u);
    addc(V[2 * B], 0u);
    add_cc(V[B], a.K[0]);
#pragma unroll
    for (int j = 1; j <= B; ++j) addc_cc(V[B + j], a.K[j]);
    addc(V[2 * B + 1], 0u);
}

// all-ones / all-zero masks without branches
MPG_DI uint32_t mask_if_nonzero(uint32_t v) { return 0u - ((v | (0u - v)) >> 31); }
MPG_DI uint32_t mask_if_equal(uint32_t a, uint32_t b) { return ~mask_if_nonzero(a ^ b); }

}  // namespace mpg
