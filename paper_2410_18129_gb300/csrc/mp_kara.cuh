// One level of Karatsuba for batched products and squares (Sec. 3):
//   A = a_l + W^h a_h, B = b_l + W^h b_h,  h = NP/2 words
//   D0 = a_l b_l,  D2 = a_h b_h,  D1 = (a_l + a_h)(b_l + b_h)
//   A*B = D0 + W^h (D1 - D0 - D2) + W^2h D2
// The three half-size products run one after the other on the whole group with
// the schoolbook block products of a half shape HS (same G, M/2 words per
// thread). a_l + a_h has h words plus a carry bit c_a; with s_a, s_b the low h
// words, D1 = s_a s_b + W^h (c_a s_b + c_b s_a) + W^2h c_a c_b. Every sum and
// difference runs across the group with the same carry-lookahead as elsewhere.
#pragma once
#include "mp_kernels.cuh"

namespace mpg {

// dst[i] = a[i] + b(i) for i < G*C (thread t owns words [t*C, t*C+C)), plus carry-in
// cin (0/1, group-uniform). Returns the carry out of the top word (group-uniform).
// b is a functor word index -> word. dst may equal a.
template <class S, int C, class BF>
MPG_DI uint32_t gadd(const Grp<S> &g, uint32_t *dst, const uint32_t *a, const BF &b, uint32_t cin) {
    constexpr int G = S::G;
    uint32_t x[C];
    lds<C>(x, a + g.t * C);
    add_cc(x[0], b(g.t * C));
#pragma unroll
    for (int j = 1; j < C; ++j) addc_cc(x[j], b(g.t * C + j));
    const uint32_t gen = addc_get();
    uint32_t all = x[0];
#pragma unroll
    for (int j = 1; j < C; ++j) all &= x[j];
    const uint64_t Gm = g.gbits(gen != 0u), Pm = g.gbits(all == 0xffffffffu);
    const uint64_t in = (Pm + ((Gm << 1) | (uint64_t)cin)) ^ Pm;
    add_word<C>(x, (uint32_t)(in >> g.t) & 1u);
    gsync();
    sts<C>(dst + g.t * C, x);
    gsync();
    return (uint32_t)(in >> G) & 1u;
}

// dst[i] = a[i] - b[i] for i < G*C; returns the borrow out of the top word.
template <class S, int C>
MPG_DI uint32_t gsub(const Grp<S> &g, uint32_t *dst, const uint32_t *a, const uint32_t *b) {
    constexpr int G = S::G;
    uint32_t x[C], y[C];
    lds<C>(x, a + g.t * C);
    lds<C>(y, b + g.t * C);
    uint32_t eq = 0u;
#pragma unroll
    for (int j = 0; j < C; ++j) eq |= x[j] ^ y[j];
    const uint32_t gen = sub_n<C>(x, y);
    const uint64_t Gm = g.gbits(gen != 0u), Pm = g.gbits(eq == 0u);
    const uint64_t bin = (Pm + (Gm << 1)) ^ Pm;
    sub_word<C>(x, (uint32_t)(bin >> g.t) & 1u);
    gsync();
    sts<C>(dst + g.t * C, x);
    gsync();
    return (uint32_t)(bin >> G) & 1u;
}

// shared-memory map of one instance (words), h = HS::NP
template <class F, class HS>
struct KaraLayout {
    static constexpr int h = HS::NP;
    static_assert(2 * h == F::NP && HS::G == F::G, "HS must be F with half the words per thread");
    static constexpr int OFF_A = 0;            // a (2h)
    static constexpr int OFF_B = 2 * h;        // b (2h)
    static constexpr int OFF_SA = 4 * h;       // a_l + a_h (h)
    static constexpr int OFF_SB = 5 * h;       // b_l + b_h (h)
    static constexpr int OFF_D = 6 * h;        // D0 | D2 (4h): the result is formed in place
    static constexpr int OFF_D1 = 10 * h;      // D1, then D1 - D0 - D2 (2h)
    static constexpr int OFF_SQ = 12 * h;      // block squares of a half product (2h)
    static constexpr int OFF_P = 14 * h;       // slot spills of the half products
    static constexpr int WORDS = (OFF_P + 2 * HS::G * (HS::M + 1) + 3) & ~3;
};

template <class F, class HS, int TPB>
__global__ void __launch_bounds__(TPB) k_kara(KArgs A) {
    using L = KaraLayout<F, HS>;
    constexpr int h = L::h, MH = HS::M;
    extern __shared__ uint4 smem4[];
    uint32_t *sm = reinterpret_cast<uint32_t *>(smem4) + (threadIdx.x / F::G) * L::WORDS;
    Grp<HS> g;
    g.sm = sm;
    g.pa = sm + L::OFF_P;
    g.t = threadIdx.x % F::G;
    g.gbase = (threadIdx.x & 31) & ~(F::G - 1);
    const size_t k = (size_t)blockIdx.x * (TPB / F::G) + threadIdx.x / F::G;
    const bool valid = k < A.batch;
    uint32_t *a = sm + L::OFF_A, *b = sm + L::OFF_B, *sa = sm + L::OFF_SA, *sb = sm + L::OFF_SB;
    uint32_t *D = sm + L::OFF_D, *D1 = sm + L::OFF_D1, *SQ = sm + L::OFF_SQ;
    {
        uint32_t x[F::M];
        gload<F::M>(x, A.a, A.layout, k, valid, g.t * F::M, A.n, A.batch);
        sts<F::M>(a + g.t * F::M, x);
        if (!A.square) {
            gload<F::M>(x, A.b, A.layout, k, valid, g.t * F::M, A.n, A.batch);
            sts<F::M>(b + g.t * F::M, x);
        }
    }
    gsync();
    const uint32_t ca = gadd<HS, MH>(g, sa, a, [&](int i) { return a[h + i]; }, 0u);
    uint32_t cb = ca;
    if (!A.square) cb = gadd<HS, MH>(g, sb, b, [&](int i) { return b[h + i]; }, 0u);
    const uint32_t *sbp = A.square ? sa : sb;
    if (A.square) {
        phase_sqr<HS>(g, a, SQ, D);               // D0 = a_l^2
        phase_sqr<HS>(g, a + h, SQ, D + 2 * h);   // D2 = a_h^2
        phase_sqr<HS>(g, sa, SQ, D1);             // D1 = s_a^2
    } else {
        phase_mul<HS>(g, a, b, D);                // D0 = a_l b_l
        phase_mul<HS>(g, a + h, b + h, D + 2 * h);   // D2 = a_h b_h
        phase_mul<HS>(g, sa, sb, D1);             // D1 = s_a s_b
    }
    // D1 <- D1 + W^h (c_a s_b + c_b s_a) + W^2h c_a c_b - D0 - D2   (2h words + top word)
    const uint32_t ma = 0u - ca, mb = 0u - cb;
    uint32_t top = gadd<HS, 2 * MH>(g, D1, D1, [&](int i) { return i >= h ? (sbp[i - h] & ma) : 0u; }, 0u);
    top += gadd<HS, 2 * MH>(g, D1, D1, [&](int i) { return i >= h ? (sa[i - h] & mb) : 0u; }, 0u);
    top += ca & cb;
    top -= gsub<HS, 2 * MH>(g, D1, D1, D);
    top -= gsub<HS, 2 * MH>(g, D1, D1, D + 2 * h);
    // result = (D2 : D0) + W^h (D1 + W^2h top)
    gadd<HS, 4 * MH>(g, D, D, [&](int i) {
        return (i >= h && i < 3 * h) ? D1[i - h] : (i == 3 * h ? top : 0u);
    }, 0u);
    uint32_t x[2 * F::M];
    lds<2 * F::M>(x, D + 2 * g.t * F::M);
    gstore<2 * F::M>(A.out, x, A.layout, k, valid, 2 * g.t * F::M, 2 * A.n, A.batch);
}

// ------------------------------------------------------------------ two levels
//
// Two levels of Karatsuba (Sec. 3): the three half-size products of the level above are
// themselves one-level Karatsuba products of quarter-size schoolbook blocks, 9 quarter
// products instead of 16. One group shape QS (G threads, MQ words per thread) serves both
// levels: QS::NP = q words per quarter, h = 2q per half, f = 4q per operand.

// out[0 .. 4q) = x * y for x, y of 2q words (one Karatsuba level over quarter products).
// Scratch: sx, sy (q words each), d1 (2q words + top), sq (2q words, block squares).
template <class QS>
MPG_DI void kara1(const Grp<QS> &g, const uint32_t *x, const uint32_t *y, bool square, uint32_t *out,
                  uint32_t *sx, uint32_t *sy, uint32_t *d1, uint32_t *sq) {
    constexpr int q = QS::NP, MQ = QS::M;
    const uint32_t cx = gadd<QS, MQ>(g, sx, x, [&](int i) { return x[q + i]; }, 0u);
    uint32_t cy = cx;
    if (!square) cy = gadd<QS, MQ>(g, sy, y, [&](int i) { return y[q + i]; }, 0u);
    const uint32_t *syp = square ? sx : sy;
    if (square) {
        phase_sqr<QS>(g, x, sq, out);
        phase_sqr<QS>(g, x + q, sq, out + 2 * q);
        phase_sqr<QS>(g, sx, sq, d1);
    } else {
        phase_mul<QS>(g, x, y, out);
        phase_mul<QS>(g, x + q, y + q, out + 2 * q);
        phase_mul<QS>(g, sx, sy, d1);
    }
    const uint32_t mx = 0u - cx, my = 0u - cy;
    uint32_t top = gadd<QS, 2 * MQ>(g, d1, d1, [&](int i) { return i >= q ? (syp[i - q] & mx) : 0u; }, 0u);
    top += gadd<QS, 2 * MQ>(g, d1, d1, [&](int i) { return i >= q ? (sx[i - q] & my) : 0u; }, 0u);
    top += cx & cy;
    top -= gsub<QS, 2 * MQ>(g, d1, d1, out);
    top -= gsub<QS, 2 * MQ>(g, d1, d1, out + 2 * q);
    gadd<QS, 4 * MQ>(g, out, out, [&](int i) {
        return (i >= q && i < 3 * q) ? d1[i - q] : (i == 3 * q ? top : 0u);
    }, 0u);
}

template <class QS>
struct Kara2Layout {
    static constexpr int q = QS::NP, h = 2 * q, f = 4 * q;
    static constexpr int OFF_A = 0;                 // a (f)
    static constexpr int OFF_B = f;                 // b (f)
    static constexpr int OFF_SA = 2 * f;            // a_l + a_h (h)
    static constexpr int OFF_SB = OFF_SA + h;       // b_l + b_h (h)
    static constexpr int OFF_D = OFF_SB + h;        // D0 | D2 (2f): the result is formed in place
    static constexpr int OFF_D1 = OFF_D + 2 * f;    // D1 (f words + top)
    static constexpr int OFF_SX = OFF_D1 + f;       // inner level: s_x, s_y (q each)
    static constexpr int OFF_SY = OFF_SX + q;
    static constexpr int OFF_ID1 = OFF_SY + q;      // inner D1 (2q)
    static constexpr int OFF_SQ = OFF_ID1 + 2 * q;  // inner block squares (2q)
    static constexpr int OFF_P = OFF_SQ + 2 * q;    // slot spills of the quarter products
    static constexpr int WORDS = (OFF_P + 2 * QS::G * (QS::M + 1) + 3) & ~3;
};

template <class QS, int TPB>
__global__ void __launch_bounds__(TPB) k_kara2(KArgs A) {
    using L = Kara2Layout<QS>;
    constexpr int q = L::q, h = L::h, G = QS::G, MQ = QS::M, MF = 4 * MQ;
    extern __shared__ uint4 smem4[];
    uint32_t *sm = reinterpret_cast<uint32_t *>(smem4) + (threadIdx.x / G) * L::WORDS;
    Grp<QS> g;
    g.sm = sm;
    g.pa = sm + L::OFF_P;
    g.t = threadIdx.x % G;
    g.gbase = (threadIdx.x & 31) & ~(G - 1);
    const size_t k = (size_t)blockIdx.x * (TPB / G) + threadIdx.x / G;
    const bool valid = k < A.batch;
    uint32_t *a = sm + L::OFF_A, *b = sm + L::OFF_B, *sa = sm + L::OFF_SA, *sb = sm + L::OFF_SB;
    uint32_t *D = sm + L::OFF_D, *D1 = sm + L::OFF_D1;
    uint32_t *sx = sm + L::OFF_SX, *sy = sm + L::OFF_SY, *id1 = sm + L::OFF_ID1, *sq = sm + L::OFF_SQ;
    {
        uint32_t x[MF];
        gload<MF>(x, A.a, A.layout, k, valid, g.t * MF, A.n, A.batch);
        sts<MF>(a + g.t * MF, x);
        if (!A.square) {
            gload<MF>(x, A.b, A.layout, k, valid, g.t * MF, A.n, A.batch);
            sts<MF>(b + g.t * MF, x);
        }
    }
    g.sync();
    const bool sqr = A.square != 0;
    const uint32_t ca = gadd<QS, 2 * MQ>(g, sa, a, [&](int i) { return a[h + i]; }, 0u);
    uint32_t cb = ca;
    if (!sqr) cb = gadd<QS, 2 * MQ>(g, sb, b, [&](int i) { return b[h + i]; }, 0u);
    const uint32_t *sbp = sqr ? sa : sb;
    kara1<QS>(g, a, b, sqr, D, sx, sy, id1, sq);                 // D0 = a_l b_l
    kara1<QS>(g, a + h, b + h, sqr, D + 2 * h, sx, sy, id1, sq); // D2 = a_h b_h
    kara1<QS>(g, sa, sbp, sqr, D1, sx, sy, id1, sq);             // D1 = s_a s_b
    const uint32_t ma = 0u - ca, mb = 0u - cb;
    uint32_t top = gadd<QS, 4 * MQ>(g, D1, D1, [&](int i) { return i >= h ? (sbp[i - h] & ma) : 0u; }, 0u);
    top += gadd<QS, 4 * MQ>(g, D1, D1, [&](int i) { return i >= h ? (sa[i - h] & mb) : 0u; }, 0u);
    top += ca & cb;
    top -= gsub<QS, 4 * MQ>(g, D1, D1, D);
    top -= gsub<QS, 4 * MQ>(g, D1, D1, D + 2 * h);
    // result = (D2 : D0) + W^h (D1 + W^2h top), in two halves of f words
    const uint32_t c = gadd<QS, 4 * MQ>(g, D, D, [&](int i) { return i >= h ? D1[i - h] : 0u; }, 0u);
    gadd<QS, 4 * MQ>(g, D + 2 * h, D + 2 * h, [&](int i) {
        return i < h ? D1[h + i] : (i == h ? top : 0u);
    }, c);
    uint32_t x[2 * MF];
    lds<2 * MF>(x, D + 2 * g.t * MF);
    gstore<2 * MF>(A.out, x, A.layout, k, valid, 2 * g.t * MF, 2 * A.n, A.batch);
}

template <class QS, int TPB>
static cudaError_t launch_kara2(const KArgs &A, cudaStream_t st) {
    using L = Kara2Layout<QS>;
    constexpr int GPB = TPB / QS::G;
    const size_t smem = (size_t)GPB * L::WORDS * 4;
    static std::atomic<unsigned long long> attr_done{0ull};
    const cudaError_t e = smem_attr_once(attr_done, k_kara2<QS, TPB>, smem);
    if (e != cudaSuccess) return e;
    const size_t blocks = (A.batch + GPB - 1) / GPB;
    k_kara2<QS, TPB><<<(unsigned)blocks, TPB, smem, st>>>(A);
    return cudaGetLastError();
}

template <class F, class HS, int TPB>
static cudaError_t launch_kara(const KArgs &A, cudaStream_t st) {
    using L = KaraLayout<F, HS>;
    constexpr int GPB = TPB / F::G;
    const size_t smem = (size_t)GPB * L::WORDS * 4;
    static std::atomic<unsigned long long> attr_done{0ull};
    const cudaError_t e = smem_attr_once(attr_done, k_kara<F, HS, TPB>, smem);
    if (e != cudaSuccess) return e;
    const size_t blocks = (A.batch + GPB - 1) / GPB;
    k_kara<F, HS, TPB><<<(unsigned)blocks, TPB, smem, st>>>(A);
    return cudaGetLastError();
}

}  // namespace mpg
