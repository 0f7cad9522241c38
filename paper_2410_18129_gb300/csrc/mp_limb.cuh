// 32-bit limb primitives: IMAD / IMAD.HI carry chains written as inline PTX.
//
// The paper's primitive is the 52-bit fused multiply-add VPMADD52 (lo and hi
// halves, Sec. 2). Its GPU counterpart is the 32x32-bit multiply-add in two
// halves, mad.lo.cc.u32 / madc.hi.cc.u32, chained through the carry flag.
// Every function here runs the same instruction sequence for every input value.
#pragma once
#include <cstdint>

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

// all-ones / all-zero masks without branches
MPG_DI uint32_t mask_if_nonzero(uint32_t v) { return 0u - ((v | (0u - v)) >> 31); }
MPG_DI uint32_t mask_if_equal(uint32_t a, uint32_t b) { return ~mask_if_nonzero(a ^ b); }

}  // namespace mpg
