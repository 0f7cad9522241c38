/*
 * Plain CPU big-integer oracle for batched Montgomery arithmetic.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * timed CPU-baseline leg of the benchmark may load this code; the product
 * path never does. It shares no code, header or table with the CUDA path.
 *
 * Values are little-endian arrays of 32-bit words (W = 2^32), n words per
 * value, R = W^n. Everything here is written to be obviously correct, not fast:
 *
 *   plain definitions (the parity targets)
 *     or_mul          C = A*B                          schoolbook (Alg. 1 "Ensure")
 *     or_mod          U mod V                          Knuth, TAOCP vol. 2, 4.3.1, Algorithm D
 *     or_neg_inv      N' = (-N)^{-1} mod R             bit-by-bit construction (Sec. 4, Alg. 3 input)
 *     or_mont_def     a*b*R^{-1} mod N                 product, remainder, 32n modular halvings
 *     or_modexp       a^e mod N                        left-to-right square-and-multiply (Alg. 7 "Ensure")
 *
 *   method model (the paper's steps, used to pin intermediates)
 *     or_montred_alg5 classical reduction q = T*N' mod R, C = (T+qN)/R        (Alg. 3 / Alg. 5)
 *     or_montred_alg6 truncated reduction: c_add, column n-1 sum, high half   (Alg. 6, Thm. 1, Thm. 2)
 *     or_montred_tkara truncated reduction, Karatsuba form: D2 in full, column
 *                     estimates of D0 and D1, carry from word n-1 of -T    (Sec. 5.1, Karatsuba)
 *     or_modexp_alg7  fixed-window left-to-right exponentiation               (Alg. 7)
 *
 * Reading adopted where the paper is silent: every Montgomery result is made
 * canonical (< N) by one conditional subtraction, since R = W^n leaves no
 * slack above N (Alg. 5 guarantees only C < 2N).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint32_t limb;
typedef uint64_t dlimb;

/* ------------------------------------------------------------------ helpers */

static int cmp_n(const limb *a, const limb *b, int n) {
    for (int i = n - 1; i >= 0; --i) {
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    }
    return 0;
}

/* a[0..n) += b[0..n), returns carry */
static limb add_n(limb *a, const limb *b, int n) {
    dlimb c = 0;
    for (int i = 0; i < n; ++i) {
        c += (dlimb)a[i] + b[i];
        a[i] = (limb)c;
        c >>= 32;
    }
    return (limb)c;
}

/* a[0..n) -= b[0..n), returns borrow */
static limb sub_n(limb *a, const limb *b, int n) {
    limb borrow = 0;
    for (int i = 0; i < n; ++i) {
        dlimb d = (dlimb)a[i] - b[i] - borrow;
        a[i] = (limb)d;
        borrow = (limb)((d >> 32) ? 1 : 0);
    }
    return borrow;
}

/* add the 64-bit value v at word position pos of a[0..len), carrying upward */
static void add_at(limb *a, int len, int pos, dlimb v) {
    while (v && pos < len) {
        dlimb s = (dlimb)a[pos] + (v & 0xffffffffu);
        a[pos] = (limb)s;
        v = (v >> 32) + (s >> 32);
        ++pos;
    }
}

static int sig_len(const limb *a, int n) {
    while (n > 0 && a[n - 1] == 0) --n;
    return n;
}

/* ------------------------------------------------------- plain definitions */

/* c[0..na+nb) = a[0..na) * b[0..nb); schoolbook, c must not alias a or b. */
void or_mul(limb *c, const limb *a, int na, const limb *b, int nb) {
    memset(c, 0, sizeof(limb) * (size_t)(na + nb));
    for (int i = 0; i < na; ++i) {
        dlimb carry = 0;
        for (int j = 0; j < nb; ++j) {
            dlimb t = (dlimb)a[i] * b[j] + c[i + j] + carry;
            c[i + j] = (limb)t;
            carry = t >> 32;
        }
        c[i + nb] = (limb)carry;
    }
}

/*
 * r[0..nv) = u[0..nu) mod v[0..nv). Knuth's Algorithm D: normalise so the top
 * divisor word has its high bit set, estimate each quotient word from the top
 * two dividend words, correct the estimate at most twice, multiply-subtract,
 * and add back on the rare negative result. Returns -1 if v == 0.
 */
int or_mod(limb *r, const limb *u, int nu, const limb *v, int nv_in) {
    int nv = sig_len(v, nv_in);
    if (nv <= 0) return -1;
    memset(r, 0, sizeof(limb) * (size_t)nv_in);
    int nus = sig_len(u, nu);
    if (nus < nv) {
        memcpy(r, u, sizeof(limb) * (size_t)nus);
        return 0;
    }
    if (nv == 1) {
        dlimb rem = 0;
        for (int i = nus - 1; i >= 0; --i) rem = ((rem << 32) | u[i]) % v[0];
        r[0] = (limb)rem;
        return 0;
    }
    int s = __builtin_clz(v[nv - 1]);
    limb *vn = (limb *)malloc(sizeof(limb) * (size_t)nv);
    limb *un = (limb *)malloc(sizeof(limb) * (size_t)(nus + 1));
    for (int i = nv - 1; i > 0; --i)
        vn[i] = s ? (v[i] << s) | (v[i - 1] >> (32 - s)) : v[i];
    vn[0] = v[0] << s;
    un[nus] = s ? u[nus - 1] >> (32 - s) : 0;
    for (int i = nus - 1; i > 0; --i)
        un[i] = s ? (u[i] << s) | (u[i - 1] >> (32 - s)) : u[i];
    un[0] = u[0] << s;

    const dlimb B = (dlimb)1 << 32;
    for (int j = nus - nv; j >= 0; --j) {
        dlimb num = ((dlimb)un[j + nv] << 32) | un[j + nv - 1];
        dlimb qhat = num / vn[nv - 1];
        dlimb rhat = num % vn[nv - 1];
        while (qhat >= B || qhat * vn[nv - 2] > ((rhat << 32) | un[j + nv - 2])) {
            --qhat;
            rhat += vn[nv - 1];
            if (rhat >= B) break;
        }
        /* un[j..j+nv] -= qhat * vn */
        dlimb carry = 0;
        limb borrow = 0;
        for (int i = 0; i < nv; ++i) {
            dlimb p = qhat * vn[i] + carry;
            carry = p >> 32;
            dlimb d = (dlimb)un[i + j] - (limb)p - borrow;
            un[i + j] = (limb)d;
            borrow = (limb)((d >> 32) ? 1 : 0);
        }
        dlimb d = (dlimb)un[j + nv] - carry - borrow;
        un[j + nv] = (limb)d;
        if (d >> 32) { /* went negative: add the divisor back once */
            dlimb c = 0;
            for (int i = 0; i < nv; ++i) {
                c += (dlimb)un[i + j] + vn[i];
                un[i + j] = (limb)c;
                c >>= 32;
            }
            un[j + nv] += (limb)c;
        }
    }
    for (int i = 0; i < nv; ++i)
        r[i] = s ? (un[i] >> s) | (un[i + 1] << (32 - s)) : un[i];
    free(vn);
    free(un);
    return 0;
}

/*
 * N' = (-N)^{-1} mod W^n for odd N. Built one bit at a time: keep
 * P = N*x + 1 mod W^n; whenever bit k of P is set, add 2^k to x (and N*2^k to
 * P), which clears bit k and leaves lower bits untouched. After 32n bits P = 0,
 * i.e. N*x = -1 mod W^n. Returns -1 for even N.
 */
int or_neg_inv(limb *x, const limb *N, int n) {
    if ((N[0] & 1u) == 0) return -1;
    limb *P = (limb *)calloc((size_t)n, sizeof(limb));
    memset(x, 0, sizeof(limb) * (size_t)n);
    P[0] = 1;
    for (int k = 0; k < 32 * n; ++k) {
        int w = k >> 5, b = k & 31;
        if ((P[w] >> b) & 1u) {
            x[w] |= 1u << b;
            /* P += N << k (mod W^n) */
            dlimb c = 0;
            for (int i = w; i < n; ++i) {
                int src = i - w;
                limb lo = N[src] << b;
                limb hi_in = (b && src > 0) ? N[src - 1] >> (32 - b) : 0;
                c += (dlimb)P[i] + (lo | hi_in);
                P[i] = (limb)c;
                c >>= 32;
            }
        }
    }
    free(P);
    return 0;
}

/* x <- x / 2 mod N for 0 <= x < N, N odd: add N first when x is odd. */
static void half_mod(limb *x, const limb *N, int n) {
    limb top = 0;
    if (x[0] & 1u) top = add_n(x, N, n);
    for (int i = 0; i < n - 1; ++i) x[i] = (x[i] >> 1) | (x[i + 1] << 31);
    x[n - 1] = (x[n - 1] >> 1) | (top << 31);
}

/* c = a * b * R^{-1} mod N with R = W^n: reduce a*b mod N, then halve 32n times. */
int or_mont_def(limb *c, const limb *a, const limb *b, const limb *N, int n) {
    if ((N[0] & 1u) == 0) return -1;
    limb *t = (limb *)malloc(sizeof(limb) * (size_t)(2 * n));
    or_mul(t, a, n, b, n);
    or_mod(c, t, 2 * n, N, n);
    for (int k = 0; k < 32 * n; ++k) half_mod(c, N, n);
    free(t);
    return 0;
}

/* R mod N and R^2 mod N (R = W^n) by long division. */
void or_r_consts(limb *r1, limb *r2, const limb *N, int n) {
    limb *u = (limb *)calloc((size_t)(2 * n + 1), sizeof(limb));
    u[n] = 1;
    or_mod(r1, u, n + 1, N, n);
    u[n] = 0;
    u[2 * n] = 1;
    or_mod(r2, u, 2 * n + 1, N, n);
    free(u);
}

/*
 * y = a^e mod N by left-to-right square-and-multiply over the ebits declared
 * exponent bits, with schoolbook products and Algorithm D remainders.
 */
int or_modexp(limb *y, const limb *a, const limb *e, int ebits, const limb *N, int n) {
    if (sig_len(N, n) == 0) return -1;
    limb *acc = (limb *)calloc((size_t)n, sizeof(limb));
    limb *base = (limb *)calloc((size_t)n, sizeof(limb));
    limb *t = (limb *)malloc(sizeof(limb) * (size_t)(2 * n));
    limb one[1] = {1};
    or_mod(base, a, n, N, n);
    or_mod(acc, one, 1, N, n);
    for (int k = ebits - 1; k >= 0; --k) {
        or_mul(t, acc, n, acc, n);
        or_mod(acc, t, 2 * n, N, n);
        if ((e[k >> 5] >> (k & 31)) & 1u) {
            or_mul(t, acc, n, base, n);
            or_mod(acc, t, 2 * n, N, n);
        }
    }
    memcpy(y, acc, sizeof(limb) * (size_t)n);
    free(acc);
    free(base);
    free(t);
    return 0;
}

/* ------------------------------------------------------------ method model */

/* q = (T mod R) * N' mod R (Alg. 5 / Alg. 6, first line) */
static void low_product_q(limb *q, const limb *T, const limb *Np, int n) {
    limb *p = (limb *)malloc(sizeof(limb) * (size_t)(2 * n));
    or_mul(p, T, n, Np, n);
    memcpy(q, p, sizeof(limb) * (size_t)n);
    free(p);
}

/* C (n limbs, canonical) from the pre-subtraction value Cpre (n+1 limbs, < 2N) */
static void final_subtract(limb *C, const limb *Cpre, const limb *N, int n) {
    /* Cpre >= N  iff  its top word is set (N < W^n) or its low n words compare >= N */
    int ge = (Cpre[n] != 0) || cmp_n(Cpre, N, n) >= 0;
    memcpy(C, Cpre, sizeof(limb) * (size_t)n);
    if (ge) sub_n(C, N, n);
}

/*
 * Classical Montgomery reduction (Alg. 5; the B_fma form of Alg. 3):
 * q = T*N' mod R, C = (T + q*N)/R. Cpre (n+1 limbs) is the value before the
 * final subtraction (< 2N when T < 4N^2); C is canonical.
 */
void or_montred_alg5(limb *C, limb *Cpre, const limb *T, const limb *N, const limb *Np, int n) {
    limb *q = (limb *)malloc(sizeof(limb) * (size_t)n);
    limb *qN = (limb *)malloc(sizeof(limb) * (size_t)(2 * n));
    limb *S = (limb *)calloc((size_t)(2 * n + 1), sizeof(limb));
    low_product_q(q, T, Np, n);
    or_mul(qN, q, n, N, n);
    memcpy(S, T, sizeof(limb) * (size_t)(2 * n));
    S[2 * n] = add_n(S, qN, 2 * n);
    memcpy(Cpre, S + n, sizeof(limb) * (size_t)(n + 1));
    final_subtract(C, Cpre, N, n);
    free(q);
    free(qN);
    free(S);
}

/*
 * Truncated Montgomery reduction (Alg. 6 with Thm. 1 and Thm. 2), 32-bit words:
 *   q      = (T mod R) * N' mod R
 *   c_add  = [T mod R != 0]                                  (Eq. c_add)
 *   L      = (-T) mod R, the known low half of q*N (T + qN = 0 mod R)
 *   S      = sum_{i+j=n-1} lo(q_i N_j) + sum_{i+j=n-2} hi(q_i N_j)   (Eq. qn)
 *   gamma  = (L[n-1] - S) mod W     carry into column n-1 from below
 *   kappa  = (S + gamma - L[n-1]) / W                         carry into column n
 *   H      = kappa + sum_{i+j>=n} lo(q_i N_j) W^{i+j-n}
 *                  + sum_{i+j>=n-1} hi(q_i N_j) W^{i+j+1-n}   (Eq. qnhat) = floor(qN/R)
 *   Cpre   = floor(T/R) + H + c_add
 * dbg (optional, n+4 words): [c_add, S lo, S hi, kappa, H[0..n]] and the pp count.
 */
void or_montred_alg6(limb *C, limb *Cpre, const limb *T, const limb *N, const limb *Np, int n,
                     limb *dbg, long *pp_count) {
    limb *q = (limb *)malloc(sizeof(limb) * (size_t)n);
    limb *L = (limb *)malloc(sizeof(limb) * (size_t)n);
    limb *H = (limb *)calloc((size_t)(n + 2), sizeof(limb));
    long pp = 0;
    low_product_q(q, T, Np, n);

    limb c_add = 0;
    for (int i = 0; i < n; ++i) c_add |= T[i];
    c_add = c_add ? 1u : 0u;

    /* L = (~T_lo + 1) mod R */
    dlimb c = 1;
    for (int i = 0; i < n; ++i) {
        c += (dlimb)(limb)~T[i];
        L[i] = (limb)c;
        c >>= 32;
    }

    dlimb S = 0;
    for (int i = 0; i < n; ++i) {
        int j = n - 1 - i;
        S += (limb)((dlimb)q[i] * N[j]);
        ++pp;
    }
    for (int i = 0; i + 1 < n; ++i) {
        int j = n - 2 - i;
        S += (limb)(((dlimb)q[i] * N[j]) >> 32);
        ++pp;
    }
    limb gamma = (limb)(L[n - 1] - (limb)S);
    dlimb kappa = (S + gamma - L[n - 1]) >> 32;

    add_at(H, n + 2, 0, kappa);
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            int k = i + j;
            if (k >= n - 1) { /* hi part lands at column k+1 >= n */
                add_at(H, n + 2, k + 1 - n, ((dlimb)q[i] * N[j]) >> 32);
                ++pp;
            }
            if (k >= n) {
                add_at(H, n + 2, k - n, (limb)((dlimb)q[i] * N[j]));
                ++pp;
            }
        }
    }
    /* Cpre = T_hi + H + c_add */
    memset(Cpre, 0, sizeof(limb) * (size_t)(n + 1));
    memcpy(Cpre, H, sizeof(limb) * (size_t)(n + 1));
    Cpre[n] += add_n(Cpre, T + n, n);
    add_at(Cpre, n + 1, 0, c_add);
    final_subtract(C, Cpre, N, n);
    if (dbg) {
        dbg[0] = c_add;
        dbg[1] = (limb)S;
        dbg[2] = (limb)(S >> 32);
        dbg[3] = (limb)kappa;
        memcpy(dbg + 4, H, sizeof(limb) * (size_t)(n + 1));
    }
    if (pp_count) *pp_count = pp;
    free(q);
    free(L);
    free(H);
}

/* sub_at: a[pos ..] -= b[0 .. nb) modulo W^len (two's complement wrap) */
static void sub_at(limb *a, int len, int pos, const limb *b, int nb) {
    dlimb borrow = 0;
    for (int i = pos; i < len; ++i) {
        dlimb d = (dlimb)a[i] - (i - pos < nb ? b[i - pos] : 0u) - borrow;
        a[i] = (limb)d;
        borrow = (d >> 32) & 1u;
    }
}

/* P = (x*y) mod W^h for x, y of h words: lo halves of the pairs with i+j < h, hi halves
   of the pairs with i+j+1 < h (h^2 half products) */
static void low_half(limb *P, const limb *x, const limb *y, int h, long *pp) {
    memset(P, 0, sizeof(limb) * (size_t)h);
    for (int i = 0; i < h; ++i)
        for (int j = 0; i + j < h; ++j) {
            dlimb p = (dlimb)x[i] * y[j];
            add_at(P, h, i + j, (limb)p);
            ++*pp;
            if (i + j + 1 < h) { add_at(P, h, i + j + 1, p >> 32); ++*pp; }
        }
}

/* x + y over h words (carry returned) */
static limb half_sum(limb *s, const limb *x, const limb *y, int h) {
    memcpy(s, x, sizeof(limb) * (size_t)h);
    return add_n(s, y, h);
}

/*
 * Column estimate of floor(x*y / W^(h-1)) for x, y of h words (the truncated half
 * product of Sec. 5.1, computed like Eq. qnhat one word lower): lo halves of the
 * pairs with i+j >= h-1 at word i+j-(h-1), hi halves of the pairs with i+j >= h-2 at
 * word i+j+1-(h-1). U (h+2 words). The omitted partial products all sit below column
 * h-1 and carry less than 2h into it, so U <= floor(xy / W^(h-1)) < U + 2h.
 */
static void trunc_est(limb *U, const limb *x, const limb *y, int h, long *pp) {
    memset(U, 0, sizeof(limb) * (size_t)(h + 2));
    for (int i = 0; i < h; ++i)
        for (int j = 0; j < h; ++j) {
            int k = i + j;
            dlimb p = (dlimb)x[i] * y[j];
            if (k >= h - 1) { add_at(U, h + 2, k - (h - 1), (limb)p); ++*pp; }
            if (k >= h - 2) { add_at(U, h + 2, k + 2 - h, p >> 32); ++*pp; }
        }
}

/*
 * Truncated Montgomery reduction with one level of Karatsuba (Sec. 5.1, the
 * Karatsuba paragraph), n = 2h words, X_l / X_h the low / high h words of X:
 *   q = (T mod R) N' mod R from the low half of a Karatsuba product only:
 *       D0' = T_l N'_l in full; of D1' = (T_l + T_h)(N'_l + N'_h) and D2' = T_h N'_h
 *       only the low h words:  q_l = D0'_l,  q_h = D0'_h + D1'_l - D0'_l - D2'_l  (mod W^h)
 *   qN = W^2h D2 + W^h (D1 - D0 - D2) + D0,  D0 = q_l N_l, D2 = q_h N_h,
 *       D1 = (q_l + q_h)(N_l + N_h) = s_q s_N + W^h (c_q s_N + c_N s_q) + W^2h c_q c_N
 *   floor(qN / R) ~ D2_l + D1_h - D0_h - D2_h + W^h D2_h   (the paper's truncated form)
 * Only D2 is formed in full; D0 and s_q s_N enter through their column estimates
 * U0, U1 (trunc_est), one word below the half boundary, so that the sum
 *   S = W D2 + U1 + W (c_q s_N + c_N s_q) + W^(h+1) c_q c_N - U0 - floor(D2 / W^(h-1))
 *       + floor(U0 / W^h)
 * estimates floor(qN / W^(n-1)) to within a few units. Word n-1 of qN is known
 * (L = (-T) mod R, Thm. 1), so the error is e = (L[n-1] - S) mod W read as a signed
 * word, and floor(qN / R) = floor((S + e) / W) exactly (the "carry evaluation" the
 * paper carries over from the schoolbook case).
 *   Cpre = floor(T / R) + floor(qN / R) + c_add.
 * dbg (optional, n+3 words): [c_add, e, H[0..n]]; pp_count: 32x32-bit half products
 * (lo or hi) of the reduction. Returns -1 for odd n, -2 if the recovered value is
 * inconsistent (an estimate outside the recoverable range).
 */
int or_montred_tkara(limb *C, limb *Cpre, const limb *T, const limb *N, const limb *Np, int n,
                     limb *dbg, long *pp_count) {
    if (n < 2 || (n & 1)) return -1;
    const int h = n / 2;
    long pp = 0;
    limb *buf = (limb *)calloc((size_t)(24 * h + 16), sizeof(limb));
    limb *D0p = buf;                 /* 2h */
    limb *sT = D0p + 2 * h;          /* h  */
    limb *sNp = sT + h;              /* h  */
    limb *P = sNp + h;               /* 2h scratch product */
    limb *q = P + 2 * h;             /* 2h */
    limb *sq = q + 2 * h;            /* h  */
    limb *sN = sq + h;               /* h  */
    limb *D2 = sN + h;               /* 2h */
    limb *U0 = D2 + 2 * h;           /* h+2 */
    limb *U1 = U0 + h + 2;           /* h+2 */
    limb *S = U1 + h + 2;            /* 2h+2 */
    limb *L = S + 2 * h + 2;         /* n  */

    /* q, low half of a Karatsuba product */
    or_mul(D0p, T, h, Np, h);
    pp += 2L * h * h;
    half_sum(sT, T, T + h, h);
    half_sum(sNp, Np, Np + h, h);
    memcpy(q, D0p, sizeof(limb) * (size_t)(2 * h));
    low_half(P, sT, sNp, h, &pp);       /* D1'_l */
    add_n(q + h, P, h);
    low_half(P, T + h, Np + h, h, &pp); /* D2'_l */
    sub_n(q + h, P, h);
    sub_n(q + h, D0p, h);

    limb c_add = 0;
    for (int i = 0; i < n; ++i) c_add |= T[i];
    c_add = c_add ? 1u : 0u;
    dlimb c = 1;                        /* L = (~T_lo + 1) mod R */
    for (int i = 0; i < n; ++i) {
        c += (dlimb)(limb)~T[i];
        L[i] = (limb)c;
        c >>= 32;
    }

    /* high half of qN */
    const limb c_q = half_sum(sq, q, q + h, h);
    const limb c_N = half_sum(sN, N, N + h, h);
    or_mul(D2, q + h, h, N + h, h);
    pp += 2L * h * h;
    trunc_est(U0, q, N, h, &pp);
    trunc_est(U1, sq, sN, h, &pp);

    memset(S, 0, sizeof(limb) * (size_t)(2 * h + 2));
    memcpy(S + 1, D2, sizeof(limb) * (size_t)(2 * h));               /* W D2 */
    for (int i = 0; i < h + 2; ++i) add_at(S, 2 * h + 2, i, U1[i]);  /* U1 */
    for (int i = 0; i < h; ++i) {                                    /* W (c_q s_N + c_N s_q) */
        if (c_q) add_at(S, 2 * h + 2, 1 + i, sN[i]);
        if (c_N) add_at(S, 2 * h + 2, 1 + i, sq[i]);
    }
    add_at(S, 2 * h + 2, h + 1, (dlimb)(c_q & c_N));                 /* W^(h+1) c_q c_N */
    sub_at(S, 2 * h + 2, 0, U0, h + 2);                              /* - U0 */
    sub_at(S, 2 * h + 2, 0, D2 + h - 1, h + 1);                      /* - floor(D2 / W^(h-1)) */
    add_at(S, 2 * h + 2, 0, U0[h]);                                  /* + floor(U0 / W^h) */
    const int32_t e = (int32_t)(L[n - 1] - S[0]);
    if (e >= 0) {
        add_at(S, 2 * h + 2, 0, (dlimb)e);
    } else {
        limb m = (limb)(-(int64_t)e);
        sub_at(S, 2 * h + 2, 0, &m, 1);
    }
    int bad = (S[0] != L[n - 1]) || S[2 * h + 1] != 0;   /* S + e must be floor(qN / W^(n-1)) >= 0 */

    /* Cpre = T_hi + H + c_add, H = S[1 .. n] */
    memset(Cpre, 0, sizeof(limb) * (size_t)(n + 1));
    memcpy(Cpre, S + 1, sizeof(limb) * (size_t)n);
    Cpre[n] = add_n(Cpre, T + n, n);
    add_at(Cpre, n + 1, 0, c_add);
    final_subtract(C, Cpre, N, n);
    if (dbg) {
        dbg[0] = c_add;
        dbg[1] = (limb)e;
        memcpy(dbg + 2, S + 1, sizeof(limb) * (size_t)(n + 1));
    }
    if (pp_count) *pp_count = pp;
    free(buf);
    return bad ? -2 : 0;
}

/* Montgomery product through one of the reductions: red 0 = Alg. 6, 1 = Alg. 5,
   3 = Alg. 6 with the truncated Karatsuba high half (Sec. 5.1; n even). */
static void mont_model(limb *C, const limb *a, const limb *b, const limb *N, const limb *Np, int n,
                       int red, limb *T, limb *Cpre) {
    or_mul(T, a, n, b, n);
    if (red == 0)
        or_montred_alg6(C, Cpre, T, N, Np, n, NULL, NULL);
    else if (red == 3)
        or_montred_tkara(C, Cpre, T, N, Np, n, NULL, NULL);
    else
        or_montred_alg5(C, Cpre, T, N, Np, n);
}

int or_mont_model(limb *C, const limb *a, const limb *b, const limb *N, int n, int red) {
    if ((N[0] & 1u) == 0 || (red == 3 && (n & 1))) return -1;
    limb *Np = (limb *)malloc(sizeof(limb) * (size_t)n);
    limb *T = (limb *)malloc(sizeof(limb) * (size_t)(2 * n));
    limb *Cpre = (limb *)malloc(sizeof(limb) * (size_t)(n + 1));
    or_neg_inv(Np, N, n);
    mont_model(C, a, b, N, Np, n, red, T, Cpre);
    free(Np);
    free(T);
    free(Cpre);
    return 0;
}

/*
 * Fixed-window left-to-right exponentiation (Alg. 7) over the model Montgomery
 * products. Table G[i] = a^i R mod N for i < 2^w (G[0] = R mod N); the exponent
 * is padded with leading zeros to ceil(ebits/w)*w bits and every window, the
 * top one included, costs w squarings and one multiplication (by G[0] when the
 * window is zero).
 */
int or_modexp_alg7(limb *y, const limb *a, const limb *e, int ebits, const limb *N, int n, int w,
                   int red) {
    if ((N[0] & 1u) == 0 || w < 1 || w > 8 || (red == 3 && (n & 1))) return -1;
    int E = 1 << w;
    limb *Np = (limb *)malloc(sizeof(limb) * (size_t)n);
    limb *R1 = (limb *)malloc(sizeof(limb) * (size_t)n);
    limb *R2 = (limb *)malloc(sizeof(limb) * (size_t)n);
    limb *G = (limb *)malloc(sizeof(limb) * (size_t)n * (size_t)E);
    limb *Y = (limb *)malloc(sizeof(limb) * (size_t)n);
    limb *Z = (limb *)malloc(sizeof(limb) * (size_t)n);
    limb *ar = (limb *)malloc(sizeof(limb) * (size_t)n);
    limb *T = (limb *)malloc(sizeof(limb) * (size_t)(2 * n));
    limb *Cpre = (limb *)malloc(sizeof(limb) * (size_t)(n + 1));
    or_neg_inv(Np, N, n);
    or_r_consts(R1, R2, N, n);
    or_mod(ar, a, n, N, n);
    memcpy(G, R1, sizeof(limb) * (size_t)n);
    if (E > 1) mont_model(G + n, ar, R2, N, Np, n, red, T, Cpre);
    for (int i = 2; i < E; ++i)
        mont_model(G + (size_t)i * n, G + (size_t)(i - 1) * n, G + n, N, Np, n, red, T, Cpre);
    memcpy(Y, R1, sizeof(limb) * (size_t)n);
    int windows = (ebits + w - 1) / w;
    for (int k = windows - 1; k >= 0; --k) {
        unsigned b = 0;
        for (int t = w - 1; t >= 0; --t) {
            int bit = k * w + t;
            unsigned v = (bit < ebits) ? (e[bit >> 5] >> (bit & 31)) & 1u : 0u;
            b = (b << 1) | v;
        }
        for (int s = 0; s < w; ++s) {
            mont_model(Z, Y, Y, N, Np, n, red, T, Cpre);
            memcpy(Y, Z, sizeof(limb) * (size_t)n);
        }
        mont_model(Z, Y, G + (size_t)b * n, N, Np, n, red, T, Cpre);
        memcpy(Y, Z, sizeof(limb) * (size_t)n);
    }
    memset(Z, 0, sizeof(limb) * (size_t)n);
    Z[0] = 1;
    mont_model(y, Y, Z, N, Np, n, red, T, Cpre);
    free(Np); free(R1); free(R2); free(G); free(Y); free(Z); free(ar); free(T); free(Cpre);
    return 0;
}

/* ------------------------------------------------------------ batch drivers */
/* Instance-major arrays: value k occupies words [k*n, (k+1)*n). nthreads <= 0: all cores. */

#ifdef _OPENMP
#include <omp.h>
#define OR_PAR _Pragma("omp parallel for schedule(dynamic, 1) num_threads(nt)")
static int threads(int nthreads) { return nthreads > 0 ? nthreads : omp_get_max_threads(); }
#else
#define OR_PAR
static int threads(int nthreads) { (void)nthreads; return 1; }
#endif

int or_threads_used(int nthreads) { return threads(nthreads); }

void or_batch_mul(limb *c, const limb *a, const limb *b, long batch, int n, int nthreads) {
    int nt = threads(nthreads);
    (void)nt;
    OR_PAR
    for (long k = 0; k < batch; ++k) or_mul(c + 2 * n * k, a + n * k, n, b + n * k, n);
}

void or_batch_sqr(limb *c, const limb *a, long batch, int n, int nthreads) {
    int nt = threads(nthreads);
    (void)nt;
    OR_PAR
    for (long k = 0; k < batch; ++k) or_mul(c + 2 * n * k, a + n * k, n, a + n * k, n);
}

int or_batch_ctx(limb *np_out, limb *r1, limb *r2, const limb *N, long batch, int n, int nthreads) {
    int nt = threads(nthreads), bad = 0;
    (void)nt;
    OR_PAR
    for (long k = 0; k < batch; ++k) {
        if (or_neg_inv(np_out + n * k, N + n * k, n)) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            bad = 1;
            continue;
        }
        or_r_consts(r1 + n * k, r2 + n * k, N + n * k, n);
    }
    return bad ? -1 : 0;
}

int or_batch_mont_def(limb *c, const limb *a, const limb *b, const limb *N, long batch, int n,
                      int nthreads) {
    int nt = threads(nthreads), bad = 0;
    (void)nt;
    OR_PAR
    for (long k = 0; k < batch; ++k)
        if (or_mont_def(c + n * k, a + n * k, b + n * k, N + n * k, n)) bad = 1;
    return bad ? -1 : 0;
}

int or_batch_mont_model(limb *c, const limb *a, const limb *b, const limb *N, long batch, int n,
                        int red, int nthreads) {
    int nt = threads(nthreads), bad = 0;
    (void)nt;
    OR_PAR
    for (long k = 0; k < batch; ++k)
        if (or_mont_model(c + n * k, a + n * k, b + n * k, N + n * k, n, red)) bad = 1;
    return bad ? -1 : 0;
}

int or_batch_modexp(limb *y, const limb *a, const limb *e, int ebits, const limb *N, long batch,
                    int n, int nthreads) {
    int ne = (ebits + 31) / 32;
    if (ne < 1) ne = 1;
    int nt = threads(nthreads), bad = 0;
    (void)nt;
    OR_PAR
    for (long k = 0; k < batch; ++k)
        if (or_modexp(y + n * k, a + n * k, e + ne * k, ebits, N + n * k, n)) bad = 1;
    return bad ? -1 : 0;
}

int or_batch_modexp_alg7(limb *y, const limb *a, const limb *e, int ebits, const limb *N,
                         long batch, int n, int w, int red, int nthreads) {
    int ne = (ebits + 31) / 32;
    if (ne < 1) ne = 1;
    int nt = threads(nthreads), bad = 0;
    (void)nt;
    OR_PAR
    for (long k = 0; k < batch; ++k)
        if (or_modexp_alg7(y + n * k, a + n * k, e + ne * k, ebits, N + n * k, n, w, red)) bad = 1;
    return bad ? -1 : 0;
}
