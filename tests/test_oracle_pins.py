"""Pins for the CPU oracle: each check ties it to something other than itself
(Python's own integer arithmetic and pow, closed forms, the paper's theorems,
brute force on tiny inputs, Fermat on generated primes)."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

W = 1 << 32


def rng(sub=0):
    return si.stream(0, "test", "other", sub)


def rand_vals(r, batch, bits):
    return si.random_bits(r, batch, bits)


# ---------------------------------------------------------------- plain products

@pytest.mark.parametrize("n", [1, 2, 3, 7, 32, 64, 129, 130])
def test_mul_sqr_match_python(n):
    r = rng(n)
    a = rand_vals(r, 16, 32 * n)
    b = rand_vals(r, 16, 32 * n)
    a[0] = 0xFFFFFFFF          # all-ones operands stress every carry
    b[0] = 0xFFFFFFFF
    a[1] = 0
    c = oracle.mul(a, b)
    s = oracle.sqr(a)
    for k in range(16):
        A, B = si.to_int(a[k]), si.to_int(b[k])
        assert si.to_int(c[k]) == A * B
        assert si.to_int(s[k]) == A * A


def test_mul_bruteforce_one_word():
    vals = np.array([0, 1, 2, 3, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFE, 0xFFFFFFFF], np.uint32)
    a = np.repeat(vals, len(vals))[:, None]
    b = np.tile(vals, len(vals))[:, None]
    c = oracle.mul(a, b)
    for k in range(a.shape[0]):
        assert si.to_int(c[k]) == int(a[k, 0]) * int(b[k, 0])


# ---------------------------------------------------------------- Algorithm D

def test_mod_matches_python_including_corrections():
    r = rng(1)
    cases = 0
    for nv in (2, 3, 5, 33, 64):
        for nu in (nv, nv + 1, 2 * nv, 2 * nv + 1):
            for trial in range(40):
                # limbs near 0 or all-ones make qhat corrections and add-back likely
                pick = r.integers(0, 4, size=nu + nv)
                pool = np.array([0, 1, 0xFFFFFFFF, 0x80000000], np.uint32)
                u = np.where(r.random(nu) < 0.5, pool[pick[:nu]],
                             r.integers(0, W, nu, dtype=np.uint64).astype(np.uint32))
                v = np.where(r.random(nv) < 0.5, pool[pick[nu:]],
                             r.integers(0, W, nv, dtype=np.uint64).astype(np.uint32))
                if not v.any():
                    v[0] = 1
                got = si.to_int(oracle.mod(u, v))
                assert got == si.to_int(u) % si.to_int(v)
                cases += 1
    assert cases > 500


def test_mod_add_back_case():
    # u = 0x7fff800000000000 (as 3 words) style case: the first quotient estimate
    # is one too large and survives the two-word test, so the add-back runs.
    u = np.array([0x00000000, 0x00000000, 0x80000000, 0x00007FFF], np.uint32)
    v = np.array([0x00000001, 0x00000000, 0x00008000], np.uint32)
    assert si.to_int(oracle.mod(u, v)) == si.to_int(u) % si.to_int(v)
    for k in range(2000):
        r = rng(100 + k)
        v = r.integers(0, W, 3, dtype=np.uint64).astype(np.uint32)
        v[2] = 0x80000000 | (v[2] & 0xFF)
        u = r.integers(0, W, 5, dtype=np.uint64).astype(np.uint32)
        u[3:] = v[1:]  # top of u close to the divisor: many corrections
        assert si.to_int(oracle.mod(u, v)) == si.to_int(u) % si.to_int(v)


# ---------------------------------------------------------------- Montgomery constants

@pytest.mark.parametrize("bits", [17, 32, 33, 64, 1024, 2048, 4108])
def test_ctx_constants(bits):
    n = si.limbs_for(bits)
    N = si.random_odd_moduli(rng(bits), 6, bits)
    Np, r1, r2 = oracle.ctx(N)
    R = 1 << (32 * n)
    for k in range(6):
        Nk = si.to_int(N[k])
        assert (si.to_int(Np[k]) * Nk) % R == R - 1
        assert si.to_int(Np[k]) == (-pow(Nk, -1, R)) % R
        assert si.to_int(r1[k]) == R % Nk
        assert si.to_int(r2[k]) == R * R % Nk


def test_ctx_rejects_even_modulus():
    with pytest.raises(ValueError):
        oracle.ctx(np.array([[4, 1]], np.uint32))


# ---------------------------------------------------------------- Montgomery products

@pytest.mark.parametrize("bits", [32, 64, 96, 1024, 2048])
def test_mont_definition_and_invariant(bits):
    n = si.limbs_for(bits)
    b = si.make_batch(0, "test", 12, bits, ebits=1, sub=bits)
    R = 1 << (32 * n)
    cdef = oracle.mont_def(b.a, b.b, b.N)
    for red in (0, 1):
        cm = oracle.mont_model(b.a, b.b, b.N, red)
        assert (cm == cdef).all()
    for k in range(12):
        Nk, ak, bk = si.to_int(b.N[k]), si.to_int(b.a[k]), si.to_int(b.b[k])
        c = si.to_int(cdef[k])
        assert c < Nk
        assert (c * R - ak * bk) % Nk == 0          # mont(x,y) * R == x*y (mod N)
        assert c == ak * bk * pow(R, -1, Nk) % Nk


def test_mont_bruteforce_tiny_moduli():
    """Exhaustive over small odd N < 2^8 (n=1, R=2^32) and all a, b < N on a grid."""
    Ns, As, Bs = [], [], []
    for N in range(3, 256, 2):
        for a in range(0, N, max(1, N // 7)):
            for b in (0, 1, N - 1, (3 * N) // 5):
                Ns.append(N)
                As.append(a)
                Bs.append(b)
    N = np.array(Ns, np.uint32)[:, None]
    a = np.array(As, np.uint32)[:, None]
    b = np.array(Bs, np.uint32)[:, None]
    R = 1 << 32
    want = [x * y * pow(R, -1, m) % m for x, y, m in zip(As, Bs, Ns)]
    for red in (0, 1):
        got = oracle.mont_model(a, b, N, red)[:, 0]
        assert [int(v) for v in got] == want
    assert [int(v) for v in oracle.mont_def(a, b, N)[:, 0]] == want


def test_mont_two_word_moduli_against_128bit():
    r = rng(7)
    N = si.random_odd_moduli(r, 64, 64)
    N[0] = [1, 0x80000000]                  # N = 2^63 + 1
    N[1] = [0xFFFFFFFF, 0xFFFFFFFF]         # N = 2^64 - 1
    a = si.uniform_below(r, N, 64)
    b = si.uniform_below(r, N, 64)
    R = 1 << 64
    for red in (0, 1):
        got = oracle.mont_model(a, b, N, red)
        for k in range(64):
            Nk = si.to_int(N[k])
            assert si.to_int(got[k]) == si.to_int(a[k]) * si.to_int(b[k]) * pow(R, -1, Nk) % Nk


# ---------------------------------------------------------------- Theorems 1 and 2

def _reduction_cases(bits, count, sub):
    """T values below N*R (< 4N^2 for a top-bit-set N, and fits 2n words) with structured
    low halves (zero, single word, dense)."""
    n = si.limbs_for(bits)
    r = rng(sub)
    N = si.random_odd_moduli(r, count, bits)
    out = []
    for k in range(count):
        Nk = si.to_int(N[k])
        mode = k % 5
        R = 1 << (32 * n)
        T = int.from_bytes(r.bytes(8 * n + 8), "little") % (Nk * R)
        if mode == 1:
            T = (T >> (32 * n)) << (32 * n)                   # T mod R == 0  -> c_add = 0
        elif mode == 2:
            T = ((T >> (32 * n)) << (32 * n)) | (1 << (32 * (n - 1)))   # only the top low word set
        elif mode == 3:
            T = ((T >> (32 * n)) << (32 * n)) | 1             # only bit 0 of the low half
        T %= Nk * R
        out.append((Nk, T, R))
    return n, N, out


@pytest.mark.parametrize("bits", [32, 64, 100, 1024, 2048])
def test_theorems_1_2_and_alg5_bound(bits):
    n, N, cases = _reduction_cases(bits, 25, bits)
    Np, _, _ = oracle.ctx(N)
    for k, (Nk, T, R) in enumerate(cases):
        Tw = si.from_int(T, 2 * n)
        d6 = oracle.montred_alg6(Tw, N[k], Np[k])
        d5 = oracle.montred_alg5(Tw, N[k], Np[k])
        q = (T % R) * si.to_int(Np[k]) % R
        qN = q * Nk
        # Thm 1: the low halves sum to 0 or R, and the carry is [T mod R != 0]
        assert (T % R) + (qN % R) in (0, R)
        assert d6["c_add"] == int(T % R != 0)
        # Thm 2: H == floor(qN / R)
        assert si.to_int(d6["H"]) == qN // R
        # Alg 5: C < 2N before the final subtraction, and C == T R^-1 mod N
        assert si.to_int(d5["Cpre"]) == (T + qN) // R < 2 * Nk
        assert si.to_int(d6["Cpre"]) == si.to_int(d5["Cpre"])
        assert si.to_int(d6["C"]) == T * pow(R, -1, Nk) % Nk == si.to_int(d5["C"])
        # column n-1 sum S and the recovered carry kappa
        S = sum((q >> (32 * i) & 0xFFFFFFFF) * (Nk >> (32 * (n - 1 - i)) & 0xFFFFFFFF) % W
                for i in range(n))
        S += sum((q >> (32 * i) & 0xFFFFFFFF) * (Nk >> (32 * (n - 2 - i)) & 0xFFFFFFFF) // W
                 for i in range(n - 1))
        assert d6["S"] == S
        # the limb of qN at column n-1 is known from T alone: it is L[n-1], L = -T mod R
        assert (qN % R) >> (32 * (n - 1)) == ((R - T % R) % R) >> (32 * (n - 1))
        # kappa is the carry into column n that is left after every pp of weight >= n-1
        qi = [(q >> (32 * i)) & 0xFFFFFFFF for i in range(n)]
        Nj = [(Nk >> (32 * j)) & 0xFFFFFFFF for j in range(n)]
        upper = sum((qi[i] * Nj[j] >> 32) << (32 * (i + j + 1 - n))
                    for i in range(n) for j in range(n) if i + j >= n - 1)
        upper += sum((qi[i] * Nj[j] & 0xFFFFFFFF) << (32 * (i + j - n))
                     for i in range(n) for j in range(n) if i + j >= n)
        assert d6["kappa"] == qN // R - upper


@pytest.mark.parametrize("n", [1, 2, 5, 32, 64])
def test_truncated_pp_count(n):
    """The truncated high half touches n(n+1)/2 lo and n(n+1)/2 + (n-1) hi half-products:
    n^2 + 2n - 1 in total (the 32-bit analogue of Table 7's count)."""
    N = si.random_odd_moduli(rng(n), 1, 32 * n)
    Np, _, _ = oracle.ctx(N)
    T = np.zeros(2 * n, np.uint32)
    T[0] = 5
    d = oracle.montred_alg6(T, N[0], Np[0])
    assert d["pp"] == n * n + 2 * n - 1


# ---------------------------------------------------------------- truncated Karatsuba (Sec. 5.1)

def _tkara_check(Nk, T, n, N_words, Np_words):
    R = 1 << (32 * n)
    h = n // 2
    d = oracle.montred_tkara(si.from_int(T, 2 * n), N_words, Np_words)
    q = (T % R) * si.to_int(Np_words) % R
    qN = q * Nk
    assert si.to_int(d["H"]) == qN // R                      # the high half, exactly
    assert abs(d["e"]) <= 2 * h + 2                          # the estimate's error bound
    assert d["c_add"] == int(T % R != 0)
    assert si.to_int(d["Cpre"]) == (T + qN) // R
    if T < Nk * R:
        assert si.to_int(d["C"]) == T * pow(R, -1, Nk) % Nk
    return d


@pytest.mark.parametrize("bits", [64, 128, 1000, 2048, 4096])
def test_truncated_karatsuba_reduction(bits):
    """Karatsuba form of the truncated reduction: only D2 in full and column estimates of
    D0 and D1; word n-1 of -T recovers the carry. H must equal floor(qN/R) (Python ints)."""
    n, N, cases = _reduction_cases(bits, 25, bits + 7)
    assert n % 2 == 0
    Np, _, _ = oracle.ctx(N)
    for k, (Nk, T, R) in enumerate(cases):
        _tkara_check(Nk, T, n, N[k], Np[k])


@pytest.mark.parametrize("n", [2, 4, 8, 64])
def test_truncated_karatsuba_extremes(n):
    """Carries of every half sum set (N = W^n - 1 gives c_N = 1; q near R gives c_q = 1),
    T = 0, 1, R, W^2n - 1 and the largest T below N*R."""
    R = 1 << (32 * n)
    Ns = [R - 1, (R >> 1) + 1, R - (1 << 32) + 1, si.to_int(si.random_odd_moduli(rng(n + 50), 1, 32 * n)[0])]
    r = rng(n + 60)
    for Nk in Ns:
        Nw = si.from_int(Nk, n)
        Np = si.from_int((-pow(Nk, -1, R)) % R, n)
        Ts = [0, 1, R, R * R - 1, Nk * R - 1, (Nk - 1) ** 2, R - 1, (R - 1) * R]
        Ts += [int.from_bytes(r.bytes(8 * n), "little") for _ in range(6)]
        for T in Ts:
            _tkara_check(Nk, T, n, Nw, Np)


@pytest.mark.parametrize("n", [2, 4, 32, 64])
def test_truncated_karatsuba_pp_count(n):
    """Half products (lo or hi) of the Karatsuba-form reduction: n^2 for q (D0' in full, the
    low halves of D1' and D2'), 2h^2 for D2 and h^2 + 2h - 1 for each column estimate,
    2n^2 + 2n - 2 in all: one fewer than the schoolbook truncated reduction's n^2 + (n^2 + 2n - 1).
    One level of Karatsuba saves nothing on the two half products; the saving is in T = A*B."""
    N = si.random_odd_moduli(rng(n + 70), 1, 32 * n)
    Np, _, _ = oracle.ctx(N)
    T = np.zeros(2 * n, np.uint32)
    T[0] = 5
    d = oracle.montred_tkara(T, N[0], Np[0])
    assert d["pp"] == 2 * n * n + 2 * n - 2
    # the schoolbook count covers the high half only (n^2 + 2n - 1); q adds n^2
    assert oracle.montred_alg6(T, N[0], Np[0])["pp"] + n * n == d["pp"] + 1
    with pytest.raises(ValueError):
        oracle.montred_tkara(np.zeros(2 * 3, np.uint32), np.array([3, 0, 1], np.uint32), np.zeros(3, np.uint32))


@pytest.mark.parametrize("bits", [256, 1024, 2048])
def test_truncated_karatsuba_products_and_modexp(bits):
    b = si.make_batch(0, "test", 8, bits, ebits=min(bits, 300), sub=bits + 11)
    R = 1 << (32 * b.n)
    got = oracle.mont_model(b.a, b.b, b.N, 3)
    assert (got == oracle.mont_def(b.a, b.b, b.N)).all()
    for k in range(8):
        Nk = si.to_int(b.N[k])
        assert si.to_int(got[k]) == si.to_int(b.a[k]) * si.to_int(b.b[k]) * pow(R, -1, Nk) % Nk
    y = oracle.modexp(b.a, b.e, b.ebits, b.N)
    for w in (1, 5):
        assert (oracle.modexp_alg7(b.a, b.e, b.ebits, b.N, w, 3) == y).all()
    with pytest.raises(ValueError):   # odd n has no half split
        oracle.mont_model(b.a[:, :3], b.b[:, :3], b.N[:, :3] | np.uint32(1), 3)


# ---------------------------------------------------------------- exponentiation

@pytest.mark.parametrize("bits", [64, 1024, 2048])
def test_modexp_matches_python_pow(bits):
    b = si.make_batch(0, "test", 8, bits, sub=bits + 1)
    y = oracle.modexp(b.a, b.e, b.ebits, b.N)
    for k in range(8):
        assert si.to_int(y[k]) == pow(si.to_int(b.a[k]), si.to_int(b.e[k]), si.to_int(b.N[k]))


def test_modexp_special_cases():
    bits = 256
    n = si.limbs_for(bits)
    Ns = [2 ** bits - 1, 2 ** (bits - 1) + 1, si.to_int(si.random_odd_moduli(rng(3), 1, bits)[0])]
    cases = []
    for Nk in Ns:
        for a in (0, 1, Nk - 1, 2):
            for e in (0, 1, 2, 2 ** bits - 1, 2 ** (bits - 1)):
                cases.append((Nk, a, e))
    N = si.from_ints([c[0] for c in cases], n)
    a = si.from_ints([c[1] for c in cases], n)
    e = si.from_ints([c[2] for c in cases], n)
    y = oracle.modexp(a, e, bits, N)
    for w in (1, 3, 5):
        for red in (0, 1):
            assert (oracle.modexp_alg7(a, e, bits, N, w, red) == y).all()
    for k, (Nk, ak, ek) in enumerate(cases):
        assert si.to_int(y[k]) == pow(ak, ek, Nk)


def test_window_width_independence():
    b = si.make_batch(0, "test", 4, 1024, sub=5)
    y = oracle.modexp(b.a, b.e, b.ebits, b.N)
    for w in range(1, 7):
        for red in (0, 1):
            assert (oracle.modexp_alg7(b.a, b.e, b.ebits, b.N, w, red) == y).all(), (w, red)


def test_modexp_short_and_odd_exponent_lengths():
    b = si.make_batch(0, "test", 6, 512, ebits=77, sub=6)
    y = oracle.modexp(b.a, b.e, 77, b.N)
    for k in range(6):
        assert si.to_int(y[k]) == pow(si.to_int(b.a[k]), si.to_int(b.e[k]), si.to_int(b.N[k]))
    assert (oracle.modexp_alg7(b.a, b.e, 77, b.N, 5, 0) == y).all()


def test_fermat_on_generated_primes():
    r = si.stream(0, "test", "prime")
    primes = [si.random_prime(r, 256) for _ in range(3)] + [si.random_prime(r, 1024)]
    for p in primes:
        assert p >> (p.bit_length() - 2) == 3        # top two bits set
        bits = p.bit_length()
        n = si.limbs_for(bits)
        N = si.from_ints([p] * 4, n)
        a = si.uniform_below(r, N, bits)
        a[a.sum(axis=1) == 0, 0] = 2
        e = si.from_ints([p - 1] * 4, n)
        y = oracle.modexp_alg7(a, e, bits, N, 5, 0)
        assert all(si.to_int(v) == 1 for v in y)
        y = oracle.modexp(a, e, bits, N)
        assert all(si.to_int(v) == 1 for v in y)


def test_edge_sizes_4108_4154():
    for bits in (4108, 4154):
        b = si.make_batch(0, "test", 2, bits, ebits=40, sub=bits)
        c = oracle.mul(b.a, b.b)
        for k in range(2):
            assert si.to_int(c[k]) == si.to_int(b.a[k]) * si.to_int(b.b[k])
        m = oracle.mont_model(b.a, b.b, b.N, 0)
        n = b.n
        R = 1 << (32 * n)
        for k in range(2):
            Nk = si.to_int(b.N[k])
            assert si.to_int(m[k]) == si.to_int(b.a[k]) * si.to_int(b.b[k]) * pow(R, -1, Nk) % Nk
