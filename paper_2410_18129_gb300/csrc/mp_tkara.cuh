// Montgomery product with one level of Karatsuba (Sec. 3) and the truncated reduction in
// its Karatsuba form (Sec. 5.1), for operands of n = 2h words. Every step runs on the
// half shape HS (G threads, MH words of a half operand each; h = G*MH):
//
//   T   = X*Y = D0 + W^h (D1 - D0 - D2) + W^2h D2             (three half products)
//   q   = T_lo N' mod R, from the low half of a Karatsuba product only:
//         D0' = T_l N'_l in full; of D1' = (T_l + T_h)(N'_l + N'_h) and D2' = T_h N'_h only
//         the low h words: q_l = D0'_l, q_h = D0'_h + D1'_l - D0'_l - D2'_l  (mod W^h)
//   qN  = W^2h D2 + W^h (D1 - D0 - D2) + D0 with D0 = q_l N_l, D2 = q_h N_h and
//         D1 = (q_l + q_h)(N_l + N_h) = s_q s_N + W^h (c_q s_N + c_N s_q) + W^2h c_q c_N.
//         Only D2 is formed in full; D0 and s_q s_N enter through column estimates U0, U1 of
//         floor(. / W^(h-1)) (phase_mulhi_est), so that
//           S = W D2 + U1 + W (c_q s_N + c_N s_q) + W^(h+1) c_q c_N - U0
//               - floor(D2 / W^(h-1)) + floor(U0 / W^h)
//         estimates floor(qN / W^(n-1)) to within a few units (the paper's truncated form
//         D2_l + D1_h - D0_h - D2_h + W^h D2_h, one word lower). Word n-1 of qN is known,
//         L = ((-T) mod R)[n-1] (Thm. 1), so e = (L - S) mod W read as a signed word gives
//         floor(qN / R) = floor((S + e) / W) exactly.
//   C   = floor(T / R) + floor(qN / R) + c_add, then the constant-time C - N select.
//
// Additions and subtractions run across the group with carry-lookahead (gadd / gsumk);
// the estimates' low words are group-uniform after the butterfly of phase_mulhi_est.
#pragma once
#include "mp_kara.cuh"

namespace mpg {

// Shared-memory map of one instance (32-bit words) for the product over half shape HS_.
// Besides the full-size operands it keeps the per-modulus half sums s_N (with its carry
// c_N) and s_N' = N'_l + N'_h mod W^h, formed once per kernel (tk_prepare).
template <class HS_>
struct KShape {
    using HS = HS_;
    static_assert(!HS::WMAP && HS::MONT_OK, "Karatsuba form: lane-mapped half shape with even MH >= 4");
    static constexpr int G = HS::G, MH = HS::M, h = HS::NP;
    static constexpr int M = 2 * MH;              // words per thread of a full operand
    static constexpr int NP = 2 * h;
    static constexpr bool WMAP = false;
    static constexpr bool MONT_OK = true;
    static constexpr int OFF_X = 0;               // operand / result
    static constexpr int OFF_Y = NP;              // operand (block squares while squaring)
    static constexpr int OFF_N = 2 * NP;          // modulus
    static constexpr int OFF_NI = 3 * NP;         // N' = (-N)^-1 mod R
    static constexpr int OFF_T = 4 * NP;          // T (2NP words)
    static constexpr int OFF_SN = 6 * NP;         // s_N = N_l + N_h mod W^h
    static constexpr int OFF_SNI = OFF_SN + h;    // s_N' = N'_l + N'_h mod W^h
    static constexpr int OFF_A = OFF_SNI + h;     // scratch (4h words), see tk_product
    static constexpr int OFF_P = OFF_A + 4 * h;   // slot spills: 2G slots of MH words + 2G top words
    static constexpr int OFF_CN = OFF_P + 2 * G * (MH + 1);   // c_N, the carry of N_l + N_h
    static constexpr int WORDS_RAW = OFF_CN + 1;
    static constexpr int BANK_RES = G < 16 ? 2 * G : 16;   // instance stride as for Shape
    static constexpr int WORDS_A = (WORDS_RAW + 3) & ~3;
    static constexpr int WORDS = WORDS_A + ((BANK_RES - WORDS_A % 32) % 32 + 32) % 32;
};

// dst[i] = (c0 + sum over k < K of term(i, k)) mod W^(G*C) for i < G*C (thread t owns words
// [t*C, t*C+C)); returns the sum divided by W^(G*C) (group-uniform). A subtraction enters as
// the complemented word ~y (over all G*C words) with its +1 in c0. Each thread adds its K
// terms with carry chains into a carry word (< K), passes that word to the next thread
// (thread 0 takes c0) and adds the one it receives; the remaining one-bit carries are resolved
// across the group with the carry-lookahead. term may read dst: every read comes before the
// first write.
template <class S, int C, int K, class TF>
MPG_DI uint32_t gsumk(const Grp<S> &g, uint32_t *dst, const TF &term, uint32_t c0) {
    constexpr int G = S::G;
    const int w0 = g.t * C;
    uint32_t x[C], y[C];
#pragma unroll
    for (int j = 0; j < C; ++j) x[j] = term(w0 + j, 0);
    uint32_t top = 0u;
#pragma unroll
    for (int k = 1; k < K; ++k) {
#pragma unroll
        for (int j = 0; j < C; ++j) y[j] = term(w0 + j, k);
        add_cc(x[0], y[0]);
#pragma unroll
        for (int j = 1; j < C; ++j) addc_cc(x[j], y[j]);
        addc(top, 0u);
    }
    const uint32_t prev = __shfl_up_sync(0xffffffffu, top, 1);
    add_cc(x[0], g.t == 0 ? c0 : prev);
#pragma unroll
    for (int j = 1; j < C; ++j) addc_cc(x[j], 0u);
    const uint32_t gen = addc_get();
    uint32_t all = x[0];
#pragma unroll
    for (int j = 1; j < C; ++j) all &= x[j];
    const uint64_t Gm = g.gbits(gen != 0u), Pm = g.gbits(all == 0xffffffffu);
    const uint64_t cin = (Pm + (Gm << 1)) ^ Pm;
    add_word<C>(x, (uint32_t)(cin >> g.t) & 1u);
    const uint32_t last = __shfl_sync(0xffffffffu, top, g.gbase + G - 1);
    gsync();
    sts<C>(dst + w0, x);
    gsync();
    return last + ((uint32_t)(cin >> G) & 1u);
}

template <class S>
MPG_DI Grp<typename S::HS> half_view(const Grp<S> &g) {
    Grp<typename S::HS> gh;
    gh.sm = g.sm;
    gh.pa = g.pa;
    gh.t = g.t;
    gh.gbase = g.gbase;
    return gh;
}

template <class S>
MPG_DI void tk_prepare(const Grp<S> &g) {
    using HS = typename S::HS;
    constexpr int h = S::h, MH = S::MH;
    const Grp<HS> gh = half_view<S>(g);
    const uint32_t *N = g.N(), *NI = g.NI();
    const uint32_t cN = gadd<HS, MH>(gh, g.sm + S::OFF_SN, N, [&](int i) { return N[h + i]; }, 0u);
    gadd<HS, MH>(gh, g.sm + S::OFF_SNI, NI, [&](int i) { return NI[h + i]; }, 0u);
    if (g.t == 0) g.sm[S::OFF_CN] = cN;
    g.sync();
}

// X <- X * Y * R^-1 mod N (X^2 * R^-1 when square), R = W^NP; Y is overwritten. With lazy,
// no final subtraction (results below 2N when 4N <= R and the inputs are below 2N).
// Scratch A (4h words) and the dead halves of X and Y carry the intermediates:
//   product:    A = [s_X | s_Y | D1 (2h)]                    (squaring: block squares in Y)
//   q:          A = [q (2h) | -],  X = [s_T | D1'_l],  Y = [D2'_l | -]
//   high half:  A = [q (2h) | D2 -> floor(qN/R) (2h)],  X = [s_q | U0 words h..2h-1],
//               Y = [U1 words h..2h-1 | -]
template <class S>
MPG_DI void tk_product(const Grp<S> &g, bool square, bool lazy) {
    using HS = typename S::HS;
    constexpr int h = S::h, MH = S::MH, NP = S::NP;
    const Grp<HS> gh = half_view<S>(g);
    uint32_t *X = g.X(), *Y = g.Y(), *T = g.T(), *A = g.sm + S::OFF_A;
    const uint32_t *N = g.N(), *NI = g.NI(), *SN = g.sm + S::OFF_SN, *SNI = g.sm + S::OFF_SNI;
    uint32_t *SA = A, *SB = A + h, *D1 = A + 2 * h;       // product
    uint32_t *Q = A, *sT = X, *L1 = X + h, *L2 = Y;       // q
    uint32_t *D2 = A + 2 * h, *sq = X, *C0 = X + h, *C1 = Y;   // high half of qN
    uint32_t ca = 0u, cb = 0u, c_add = 0u, L = 0u, cq = 0u, z0 = 0u, z1 = 0u;

    // The nine half products run from one loop, so each kind of product (full, square, low
    // half, column estimate) and each step between them is inlined once:
    //   0 D0 = X_l Y_l   1 D2 = X_h Y_h   2 D1 = s_X s_Y          (squares when squaring)
    //   3 D0' = T_l N'_l   4 D1'_l = s_T s_N' mod W^h   5 D2'_l = T_h N'_h mod W^h
    //   6 D2 = q_h N_h   7 U0 ~ q_l N_l / W^(h-1)   8 U1 ~ s_q s_N / W^(h-1)
    MPG_BLOCK_LOOP
    for (int st = 0; st < 9; ++st) {
        if (st == 0) {
            ca = gadd<HS, MH>(gh, SA, X, [&](int i) { return X[h + i]; }, 0u);
            cb = ca;
            if (!square) cb = gadd<HS, MH>(gh, SB, Y, [&](int i) { return Y[h + i]; }, 0u);
        } else if (st == 3) {
            // T[h .. 4h) += D1 + W^h (c_a s_b + c_b s_a) + W^2h c_a c_b - D0 - D2   (one pass, mod
            // W^3h; the middle term is >= 0 and T < W^4h, so the window holds the exact words)
            const uint32_t *sbp = square ? SA : SB;
            const uint32_t ma = 0u - ca, mb = 0u - cb, cc = ca & cb;
            uint32_t *TW = T + h;
            gsumk<HS, 3 * MH, 6>(gh, TW, [&](int j, int k) -> uint32_t {
                switch (k) {
                    case 0: return TW[j];
                    case 1: return j < 2 * h ? D1[j] : 0u;
                    case 2: return (j >= h && j < 2 * h) ? (sbp[j - h] & ma) : (j == 2 * h ? cc : 0u);
                    case 3: return (j >= h && j < 2 * h) ? (SA[j - h] & mb) : 0u;
                    case 4: return j < 2 * h ? ~T[j] : 0xffffffffu;            // - D0
                    default: return j < 2 * h ? ~T[2 * h + j] : 0xffffffffu;   // - D2
                }
            }, 2u);
            // c_add = [T mod R != 0], low_zero = [T mod W^(NP-1) == 0], L = ((-T) mod R)[NP-1]
            uint32_t nz_all = 0u, nz_low = 0u;
            {
                uint32_t x[S::M];
                lds<S::M>(x, T + g.t * S::M);
#pragma unroll
                for (int j = 0; j < S::M; ++j) {
                    nz_all |= x[j];
                    if (g.t * S::M + j < NP - 1) nz_low |= x[j];
                }
            }
            const bool pr[2] = {nz_all != 0u, nz_low != 0u};
            uint32_t mk[2];
            g.template bits<2>(pr, mk);
            c_add = mk[0] ? 1u : 0u;
            L = ~T[NP - 1] + (mk[1] ? 0u : 1u);
        } else if (st == 4) {
            gadd<HS, MH>(gh, sT, T, [&](int i) { return T[h + i]; }, 0u);
        } else if (st == 6) {
            gsumk<HS, MH, 4>(gh, Q + h, [&](int j, int k) -> uint32_t {   // q_h = D0'_h + D1'_l - D0'_l - D2'_l
                switch (k) {
                    case 0: return Q[h + j];
                    case 1: return L1[j];
                    case 2: return ~Q[j];
                    default: return ~L2[j];
                }
            }, 2u);
            cq = gadd<HS, MH>(gh, sq, Q, [&](int i) { return Q[h + i]; }, 0u);
        }
        const uint32_t *x, *y;
        uint32_t *o;
        switch (st) {
            case 0: x = X; y = Y; o = T; break;
            case 1: x = X + h; y = Y + h; o = T + 2 * h; break;
            case 2: x = SA; y = SB; o = D1; break;
            case 3: x = T; y = NI; o = Q; break;
            case 4: x = sT; y = SNI; o = L1; break;
            case 5: x = T + h; y = NI + h; o = L2; break;
            case 6: x = Q + h; y = N + h; o = D2; break;
            case 7: x = Q; y = N; o = C0; break;
            default: x = sq; y = SN; o = C1; break;
        }
        if (st < 3 && square) {
            phase_sqr<HS>(gh, x, Y, o);          // block squares in Y (free while squaring)
        } else if (st < 4 || st == 6) {
            phase_mul<HS>(gh, x, y, o);
        } else if (st < 6) {
            phase_mullo<HS>(gh, x, y, o);
        } else {
            const uint32_t z = phase_mulhi_est<HS>(gh, x, y, o);
            if (st == 7) z0 = z;
            else z1 = z;
        }
    }

    const uint32_t cN = g.sm[S::OFF_CN];
    // word n-1 of S (before the error correction) and the carry the correction leaves
    const int64_t xs = (int64_t)z1 - (int64_t)z0 - (int64_t)D2[h - 1] + (int64_t)C0[h - 1];
    const int32_t e = (int32_t)(L - (uint32_t)xs);
    const int64_t delta = (xs + (int64_t)e - (int64_t)L) >> 32;   // exact: xs + e = L (mod W)
    // C = floor(T / R) + floor(qN / R) + c_add in one pass, with
    //   floor(qN / R) = D2 - D2_h + U1_hi - U0_hi + c_q s_N + c_N s_q + W^h c_q c_N + delta.
    // The two complemented terms add 2 R and a negative delta (sign-extended) one more R to
    // the sum; the carry out of C is what is left above them.
    const uint32_t mq = 0u - cq, mN = 0u - cN;
    const uint32_t dlo = (uint32_t)delta, dhi = delta < 0 ? 0xffffffffu : 0u;
    const uint32_t tot = gsumk<HS, 2 * MH, 8>(gh, X, [&](int i, int k) -> uint32_t {
        switch (k) {
            case 0: return T[2 * h + i];
            case 1: return D2[i];
            case 2: return i < h ? ~D2[h + i] : 0xffffffffu;
            case 3: return i < h ? C1[i] : 0u;
            case 4: return i < h ? ~C0[i] : 0xffffffffu;
            case 5: return i < h ? (SN[i] & mq) : 0u;
            case 6: return i < h ? (sq[i] & mN) : (i == h ? (cq & cN) : 0u);
            default: return i == 0 ? dlo : dhi;
        }
    }, 2u + c_add);
    const uint32_t carry = tot - 2u - (delta < 0 ? 1u : 0u);
    if (!lazy) cond_sub<S>(g, X, carry, N, X);
}

template <class HS, int TPB>
struct TKaraImpl {
    using KS = KShape<HS>;
    static cudaError_t mont(const KArgs &A, cudaStream_t st) { return launch_k<KS, TPB, 7>(k_mont<KS, TPB, 3>, A, st); }
    static cudaError_t modexp(const KArgs &A, cudaStream_t st) {
        return launch_k<KS, TPB, 8>(k_modexp<KS, TPB, 3>, A, st);
    }
    static int residency(int red) {
        if (red != 0) return -1;
        return resident_instances(k_modexp<KS, TPB, 3>, TPB, (size_t)(TPB / KS::G) * KS::WORDS * 4, TPB / KS::G);
    }
    static ShapeOps ops() {
        return ShapeOps{KS::G, KS::M, KS::NP, TPB, (size_t)(TPB / KS::G) * KS::WORDS * 4, nullptr, &mont, &modexp,
                        nullptr, &residency, nullptr, MPG_DBG_TAKE};
    }
};

}  // namespace mpg

// Montgomery products and exponentiation of the size class with padded size NP (= 2*G*MH
// words) in the Karatsuba form, over the half shape (G, MH)
#define MPG_DEFINE_TKARA(NP, G, MH, TPB)                                                      \
    namespace mpg {                                                                           \
    ShapeOps tkara_ops_##NP() { return TKaraImpl<Shape<G, MH>, TPB>::ops(); }                 \
    }
