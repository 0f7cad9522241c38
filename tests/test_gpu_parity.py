"""GPU parity: every entry point through the C ABI, compared word for word with the
CPU oracle on the same seeded inputs (integer results: bit-exact, tolerance 0)."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mp():
    import paper_2410_18129_gb300 as mp
    assert torch.cuda.is_available()
    return mp


IM, IL = 0, 1


def dev(mp, x, layout):
    """[batch, w] numpy -> device tensor in `layout`."""
    flat = x.reshape(-1) if layout == IM else mp.interleave(x)
    return mp.to_device(flat)


def host(mp, t, batch, w, layout):
    a = mp.to_host(t)
    return a.reshape(batch, w) if layout == IM else mp.deinterleave(a, batch, w)


def out_tensor(mp, batch, w, layout):
    return torch.zeros(mp.array_words(layout, batch, w), dtype=torch.int32, device="cuda")


def assert_equal(got, want, what):
    bad = np.nonzero((got != want).any(axis=1))[0]
    assert bad.size == 0, f"{what}: {bad.size} instances differ, first {bad[:8]}"


SIZES = [64, 100, 256, 512, 1000, 1024, 1500, 2048, 2500, 3072, 3500, 4000, 4096, 4108, 4154]


# ------------------------------------------------------------------ products

@pytest.mark.parametrize("bits", SIZES)
@pytest.mark.parametrize("layout", [IM, IL])
def test_mp_mul_sqr(mp, bits, layout):
    batch = 37 if bits > 3000 else 301          # ragged: several blocks plus a partial one
    b = si.make_batch(0, "test", batch, bits, ebits=1, sub=bits)
    n = b.n
    a_np = si.random_bits(si.stream(0, "test", "other", bits), batch, bits)
    a_np[0] = 0xFFFFFFFF                         # the largest bits-bit value
    if bits % 32:
        a_np[0, n - 1] = (1 << (bits % 32)) - 1
    a_np[1] = 0
    A = dev(mp, a_np, layout)
    B = dev(mp, b.b, layout)
    C = out_tensor(mp, batch, 2 * n, layout)
    mp.mp_mul(C, A, B, batch, bits, layout)
    assert_equal(host(mp, C, batch, 2 * n, layout), oracle.mul(a_np, b.b), f"mp_mul {bits}")
    mp.mp_sqr(C, A, batch, bits, layout)
    assert_equal(host(mp, C, batch, 2 * n, layout), oracle.sqr(a_np), f"mp_sqr {bits}")


def test_mp_mul_single_instance_and_tiny(mp):
    for bits in (32, 33, 64):
        x = si.random_bits(si.stream(0, "test", "other", 7), 1, bits)
        y = si.random_bits(si.stream(0, "test", "other", 8), 1, bits)
        n = x.shape[1]
        C = out_tensor(mp, 1, 2 * n, IM)
        mp.mp_mul(C, dev(mp, x, IM), dev(mp, y, IM), 1, bits, IM)
        assert_equal(host(mp, C, 1, 2 * n, IM), oracle.mul(x, y), "tiny mul")


# ------------------------------------------------------------------ Montgomery context

@pytest.mark.parametrize("bits", [64, 100, 1024, 2048, 4108])
@pytest.mark.parametrize("layout", [IM, IL])
def test_ctx_constants(mp, bits, layout):
    batch = 45
    N = si.random_odd_moduli(si.stream(0, "test", "modulus", bits), batch, bits)
    N[0] = 0xFFFFFFFF
    if bits % 32:
        N[0, -1] &= np.uint32((1 << (bits % 32)) - 1)
    ctx = mp.MontCtx(dev(mp, N, layout), batch, bits, layout)
    Np, r1, r2 = oracle.ctx(N)
    n = N.shape[1]
    assert_equal(host(mp, ctx.export(0), batch, n, layout), Np, "N'")
    assert_equal(host(mp, ctx.export(1), batch, n, layout), r1, "R mod N")
    assert_equal(host(mp, ctx.export(2), batch, n, layout), r2, "R^2 mod N")
    assert_equal(host(mp, ctx.export(3), batch, n, layout), N, "N")
    ctx.free()


def test_ctx_even_modulus_reports_first_index(mp):
    N = si.random_odd_moduli(si.stream(0, "test", "modulus", 1), 10, 1024)
    N[6, 0] &= np.uint32(0xFFFFFFFE)
    N[8, 0] &= np.uint32(0xFFFFFFFE)
    with pytest.raises(mp.MpError) as e:
        mp.MontCtx(dev(mp, N, IM), 10, 1024, IM)
    assert e.value.status == -3 and e.value.bad_index == 6


# ------------------------------------------------------------------ Montgomery products

@pytest.mark.parametrize("bits", [64, 100, 512, 1000, 1024, 2048, 3072, 4096, 4108, 4154])
@pytest.mark.parametrize("layout", [IM, IL])
def test_mont_mul_sqr(mp, bits, layout):
    batch = 29 if bits > 3000 else 203
    b = si.make_batch(0, "test", batch, bits, ebits=1, sub=1000 + bits)
    b.a[0] = 0
    b.a[1] = b.N[1] - np.array([1] + [0] * (b.n - 1), np.uint32)   # N-1 (N odd, no borrow)
    b.b[1] = b.a[1]
    n = b.n
    ctx = mp.MontCtx(dev(mp, b.N, layout), batch, bits, layout)
    A, B = dev(mp, b.a, layout), dev(mp, b.b, layout)
    C = out_tensor(mp, batch, n, layout)
    want_mul = oracle.mont_def(b.a, b.b, b.N)
    want_sqr = oracle.mont_def(b.a, b.a, b.N)
    for red in (mp.RED_TRUNCATED, mp.RED_FULL, mp.RED_CIOS):
        mp.mont_mul(C, A, B, ctx, red)
        assert_equal(host(mp, C, batch, n, layout), want_mul, f"mont_mul {bits} red={red}")
        mp.mont_sqr(C, A, ctx, red)
        assert_equal(host(mp, C, batch, n, layout), want_sqr, f"mont_sqr {bits} red={red}")
    ctx.free()


def test_mont_mul_in_place(mp):
    bits, batch = 2048, 64
    b = si.make_batch(0, "test", batch, bits, ebits=1, sub=77)
    ctx = mp.MontCtx(dev(mp, b.N, IL), batch, bits, IL)
    A, B = dev(mp, b.a, IL), dev(mp, b.b, IL)
    mp.mont_mul(A, A, B, ctx)
    assert_equal(host(mp, A, batch, b.n, IL), oracle.mont_def(b.a, b.b, b.N), "in place")


def test_mont_special_moduli(mp):
    """N = 2^t - 1 and N = 2^(t-1) + 1 with the extreme operands."""
    bits = 2048
    n = 64
    Ns = [2 ** bits - 1, 2 ** (bits - 1) + 1]
    rows = []
    for N in Ns:
        for a, bb in ((0, 0), (1, 1), (N - 1, N - 1), (N - 1, 1), (N // 2, N // 3)):
            rows.append((N, a, bb))
    N = si.from_ints([r[0] for r in rows], n)
    a = si.from_ints([r[1] for r in rows], n)
    bb = si.from_ints([r[2] for r in rows], n)
    B = len(rows)
    ctx = mp.MontCtx(dev(mp, N, IM), B, bits, IM)
    C = out_tensor(mp, B, n, IM)
    for red in (0, 1, 2):
        mp.mont_mul(C, dev(mp, a, IM), dev(mp, bb, IM), ctx, red)
        assert_equal(host(mp, C, B, n, IM), oracle.mont_def(a, bb, N), f"special red={red}")


# ------------------------------------------------------------------ exponentiation

@pytest.mark.parametrize("bits,batch,window", [(1024, 8, 5), (1024, 67, 4), (2048, 40, 5), (512, 100, 3),
                                               (100, 50, 2), (4096, 6, 6), (3072, 6, 5), (4108, 3, 5)])
@pytest.mark.parametrize("layout", [IM, IL])
def test_modexp(mp, bits, batch, window, layout):
    b = si.make_batch(0, "test", batch, bits, sub=2000 + bits)
    ctx = mp.MontCtx(dev(mp, b.N, layout), batch, bits, layout)
    Y = out_tensor(mp, batch, b.n, layout)
    want = oracle.modexp(b.a, b.e, b.ebits, b.N)
    for red in (0, 1, 2):
        mp.modexp_consttime(Y, dev(mp, b.a, layout), dev(mp, b.e, layout), b.ebits, ctx, window, red)
        assert_equal(host(mp, Y, batch, b.n, layout), want, f"modexp {bits} w={window} red={red}")


@pytest.mark.parametrize("bits", [254, 255, 1022, 1023, 2046, 4108, 4606, 4607])
def test_modexp_lazy_slack_boundary(mp, bits):
    """Sizes on both sides of 4N <= W^NP, where the exponentiation keeps products below 2N
    without the final subtraction (lazy reduction) and canonicalises once at the end:
    largest moduli, bases N-1 and N-2, all-ones exponents, random ones; both reductions."""
    n = (bits + 31) // 32
    r = si.stream(0, "test", "other", 7000 + bits)
    Ns = [2 ** bits - 1, 2 ** (bits - 1) + 1] + [si.to_int(v) for v in si.random_odd_moduli(r, 4, bits)]
    rows = []
    for N in Ns:
        for a in (N - 1, N - 2, 3):
            for e in (2 ** bits - 1, si.to_int(si.random_bits(r, 1, bits)[0])):
                rows.append((N, a, e))
    B = len(rows)
    N = si.from_ints([x[0] for x in rows], n)
    a = si.from_ints([x[1] for x in rows], n)
    e = si.from_ints([x[2] for x in rows], n)
    ctx = mp.MontCtx(dev(mp, N, IL), B, bits, IL)
    want = [pow(x[1], x[2], x[0]) for x in rows]
    for red in (0, 1, 2):
        Y = out_tensor(mp, B, n, IL)
        mp.modexp_consttime(Y, dev(mp, a, IL), dev(mp, e, IL), bits, ctx, 5, red)
        got = host(mp, Y, B, n, IL)
        bad = [k for k in range(B) if si.to_int(got[k]) != want[k]]
        assert not bad, f"{bits} bits red={red}: {len(bad)} wrong, first {bad[:4]}"
    # resident tables + fixed-base requests use the same products
    tables = torch.empty(mp.modexp_table_bytes(ctx, 4) // 4, dtype=torch.int32, device="cuda")
    mp.modexp_table_build(tables, dev(mp, a, IL), ctx, 4)
    index = np.arange(B, dtype=np.uint32)[::-1].copy()
    Y = out_tensor(mp, B, n, IL)
    mp.modexp_fixed_base(Y, mp.to_device(index), dev(mp, e[index], IL), bits, B, ctx, tables, 4)
    got = host(mp, Y, B, n, IL)
    assert all(si.to_int(got[k]) == want[index[k]] for k in range(B)), f"{bits} bits, fixed base"


def test_modexp_window_independence_and_workspace(mp):
    bits, batch = 1024, 33
    b = si.make_batch(0, "test", batch, bits, sub=31)
    ctx = mp.MontCtx(dev(mp, b.N, IL), batch, bits, IL)
    want = oracle.modexp(b.a, b.e, b.ebits, b.N)
    A, E = dev(mp, b.a, IL), dev(mp, b.e, IL)
    for w in range(1, 7):
        ws = torch.empty(mp.modexp_workspace_bytes(batch, bits, w) // 4, dtype=torch.int32, device="cuda")
        Y = out_tensor(mp, batch, b.n, IL)
        mp.modexp_consttime(Y, A, E, bits, ctx, w, workspace=ws)
        assert_equal(host(mp, Y, batch, b.n, IL), want, f"w={w}")
    small = torch.empty(16, dtype=torch.int32, device="cuda")
    with pytest.raises(mp.MpError):
        mp.modexp_consttime(Y, A, E, bits, ctx, 5, workspace=small)


def test_modexp_special_cases(mp):
    bits = 1024
    n = 32
    N1 = si.to_int(si.random_odd_moduli(si.stream(0, "test", "modulus", 5), 1, bits)[0])
    rows = []
    for N in (N1, 2 ** bits - 1, 2 ** (bits - 1) + 1):
        for a in (0, 1, N - 1, 2):
            for e in (0, 1, 2, 2 ** bits - 1, 2 ** (bits - 1)):
                rows.append((N, a, e))
    B = len(rows)
    N = si.from_ints([r[0] for r in rows], n)
    a = si.from_ints([r[1] for r in rows], n)
    e = si.from_ints([r[2] for r in rows], n)
    ctx = mp.MontCtx(dev(mp, N, IM), B, bits, IM)
    Y = out_tensor(mp, B, n, IM)
    mp.modexp_consttime(Y, dev(mp, a, IM), dev(mp, e, IM), bits, ctx, 5)
    got = host(mp, Y, B, n, IM)
    for k, (Nk, ak, ek) in enumerate(rows):
        assert si.to_int(got[k]) == pow(ak, ek, Nk), (k, hex(Nk)[:10], ak == Nk - 1, ek)
    # exponent of 0 declared bits: every result is 1 mod N
    mp.modexp_consttime(Y, dev(mp, a, IM), dev(mp, e, IM), 0, ctx, 5)
    assert all(si.to_int(v) == 1 for v in host(mp, Y, B, n, IM))


def test_modexp_short_exponents(mp):
    bits, batch = 2048, 20
    for ebits in (1, 31, 32, 33, 77, 160):
        b = si.make_batch(0, "test", batch, bits, ebits=ebits, sub=ebits)
        ctx = mp.MontCtx(dev(mp, b.N, IL), batch, bits, IL)
        Y = out_tensor(mp, batch, b.n, IL)
        mp.modexp_consttime(Y, dev(mp, b.a, IL), dev(mp, b.e, IL), ebits, ctx, 5)
        assert_equal(host(mp, Y, batch, b.n, IL), oracle.modexp(b.a, b.e, ebits, b.N), f"ebits={ebits}")


def test_fermat_on_generated_primes(mp):
    r = si.stream(0, "test", "prime", 3)
    primes = [si.random_prime(r, 1024) for _ in range(4)]
    n = 32
    N = si.from_ints(primes * 4, n)
    a = si.uniform_below(r, N, 1024)
    e = si.from_ints([p - 1 for p in primes * 4], n)
    B = N.shape[0]
    ctx = mp.MontCtx(dev(mp, N, IM), B, 1024, IM)
    Y = out_tensor(mp, B, n, IM)
    mp.modexp_consttime(Y, dev(mp, a, IM), dev(mp, e, IM), 1024, ctx, 5)
    assert all(si.to_int(v) == 1 for v in host(mp, Y, B, n, IM))


# ------------------------------------------------------------------ layout conversion

@pytest.mark.parametrize("w", [1, 3, 4, 64, 129])
def test_convert_round_trip(mp, w):
    batch = 77
    x = si.random_bits(si.stream(0, "test", "other", w), batch, 32 * w)
    src = dev(mp, x, IM)
    mid = out_tensor(mp, batch, w, IL)
    back = out_tensor(mp, batch, w, IM)
    mp.mp_convert(mid, IL, src, IM, batch, w)
    got, want = mp.to_host(mid), mp.interleave(x)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, f"{bad.size} words differ, first at {bad[:6]}: got {got[bad[:6]]} want {want[bad[:6]]}"
    mp.mp_convert(back, IM, mid, IL, batch, w)
    assert (mp.to_host(back).reshape(batch, w) == x).all()


# ------------------------------------------------------------------ one-level Karatsuba

@pytest.mark.parametrize("bits", [520, 1000, 1024, 1500, 2048, 2078, 2500, 3072, 3500, 4000, 4096, 4108, 4154])
@pytest.mark.parametrize("layout", [IM, IL])
def test_karatsuba_mul_sqr(mp, bits, layout):
    batch = 45 if bits > 3000 else 173
    a_np = si.random_bits(si.stream(0, "test", "other", 5000 + bits), batch, bits)
    b_np = si.random_bits(si.stream(0, "test", "other", 6000 + bits), batch, bits)
    n = a_np.shape[1]
    a_np[0] = 0xFFFFFFFF                        # all-ones: the half sums carry out
    b_np[0] = 0xFFFFFFFF
    if bits % 32:
        a_np[0, n - 1] = (1 << (bits % 32)) - 1
        b_np[0, n - 1] = (1 << (bits % 32)) - 1
    a_np[1] = 0
    A, B = dev(mp, a_np, layout), dev(mp, b_np, layout)
    C = out_tensor(mp, batch, 2 * n, layout)
    mp.mp_mul(C, A, B, batch, bits, layout, mp.ALGO_KARATSUBA)
    assert_equal(host(mp, C, batch, 2 * n, layout), oracle.mul(a_np, b_np), f"karatsuba mul {bits}")
    mp.mp_sqr(C, A, batch, bits, layout, mp.ALGO_KARATSUBA)
    assert_equal(host(mp, C, batch, 2 * n, layout), oracle.sqr(a_np), f"karatsuba sqr {bits}")


@pytest.mark.parametrize("shape", [(16, 8), (8, 16)])
def test_products_each_4096_bit_shape(mp, shape):
    """Schoolbook and one-level Karatsuba products on each compiled shape of the 4096-bit class
    (role-swapped: 16 roles x 8 words with half products of 16 x 4, and 8 x 16 with halves of
    8 x 8), against the oracle; all-ones operands make both half sums carry out."""
    bits, batch = 4096, 70
    a_np = si.random_bits(si.stream(0, "test", "other", 7100), batch, bits)
    b_np = si.random_bits(si.stream(0, "test", "other", 7101), batch, bits)
    a_np[0] = b_np[0] = 0xFFFFFFFF
    a_np[1] = 0
    a_np[2, :64] = 0xFFFFFFFF                    # only the low half all ones
    b_np[3, 64:] = 0xFFFFFFFF                    # only the high half all ones
    saved = mp.tune_get(bits)
    try:
        mp.tune_set(bits, *shape)
        for layout in (IM, IL):
            A, B = dev(mp, a_np, layout), dev(mp, b_np, layout)
            C = out_tensor(mp, batch, 256, layout)
            for algo in (mp.ALGO_SCHOOLBOOK, mp.ALGO_KARATSUBA):
                mp.mp_mul(C, A, B, batch, bits, layout, algo)
                assert_equal(host(mp, C, batch, 256, layout), oracle.mul(a_np, b_np), f"mul {shape} {algo}")
                mp.mp_sqr(C, A, batch, bits, layout, algo)
                assert_equal(host(mp, C, batch, 256, layout), oracle.sqr(a_np), f"sqr {shape} {algo}")
    finally:
        mp.tune_set(bits, saved["G"], saved["M"], saved["window"], saved["karatsuba_from_bits"])


def test_karatsuba_auto_and_small_sizes(mp):
    bits, batch = 4096, 9
    x = si.random_bits(si.stream(0, "test", "other", 77), batch, bits)
    C = out_tensor(mp, batch, 2 * 128, IM)
    mp.mp_mul(C, dev(mp, x, IM), dev(mp, x, IM), batch, bits, IM, mp.ALGO_AUTO)
    assert_equal(host(mp, C, batch, 256, IM), oracle.sqr(x), "auto 4096")
    y = si.random_bits(si.stream(0, "test", "other", 79), batch, 4154)
    C2 = out_tensor(mp, batch, 2 * 130, IM)
    mp.mp_sqr(C2, dev(mp, y, IM), batch, 4154, IM, mp.ALGO_AUTO)
    assert_equal(host(mp, C2, batch, 260, IM), oracle.sqr(y), "auto 4154")
    small = si.random_bits(si.stream(0, "test", "other", 78), 4, 256)
    with pytest.raises(mp.MpError) as e:
        mp.mp_mul(out_tensor(mp, 4, 16, IM), dev(mp, small, IM), dev(mp, small, IM), 4, 256, IM,
                  mp.ALGO_KARATSUBA)
    assert e.value.status == -7


# ------------------------------------------------------------------ truncated Karatsuba form (Sec. 5.1)

TKARA_SIZES = [257, 512, 513, 1000, 1024, 1025, 1500, 2046, 2048, 2100, 3072, 3073, 3500, 4094, 4096]


def _tkara_batch(bits, batch, sub):
    """Random instances plus the extremes: N = 2^bits - 1 (its halves' sum carries), operands
    0, 1, N-1 and all-ones-like values, exponent 0 and all ones."""
    b = si.make_batch(0, "test", batch, bits, sub=sub)
    n = b.n
    N0 = 2 ** bits - 1
    b.N[0] = si.from_int(N0, n)
    b.a[0] = si.from_int(N0 - 1, n)
    b.b[0] = si.from_int(N0 - 1, n)
    b.N[1] = si.from_int(2 ** (bits - 1) + 1, n)
    b.a[1] = si.from_int(1, n)
    b.b[1] = si.from_int(2 ** (bits - 1), n)
    b.a[2] = 0
    b.e[3] = 0
    b.e[4] = si.from_int(2 ** bits - 1, n)
    return b


@pytest.mark.parametrize("bits", TKARA_SIZES)
@pytest.mark.parametrize("layout", [IM, IL])
def test_truncated_karatsuba_mont(mp, bits, layout):
    """mont_mul / mont_sqr with MP_ALGO_KARATSUBA (T by one Karatsuba level, q from the low half
    of a Karatsuba product, the high half of qN in the truncated Karatsuba form) against the
    plain definition; several blocks of instances plus a ragged one."""
    batch = 83 if bits > 3000 else 203
    b = _tkara_batch(bits, batch, 8100 + bits)
    n = b.n
    ctx = mp.MontCtx(dev(mp, b.N, layout), batch, bits, layout)
    A, B = dev(mp, b.a, layout), dev(mp, b.b, layout)
    C = out_tensor(mp, batch, n, layout)
    mp.mont_mul(C, A, B, ctx, mp.RED_TRUNCATED, mp.ALGO_KARATSUBA)
    assert_equal(host(mp, C, batch, n, layout), oracle.mont_def(b.a, b.b, b.N), f"tkara mont_mul {bits}")
    mp.mont_sqr(C, A, ctx, mp.RED_TRUNCATED, mp.ALGO_KARATSUBA)
    assert_equal(host(mp, C, batch, n, layout), oracle.mont_def(b.a, b.a, b.N), f"tkara mont_sqr {bits}")
    ctx.free()


@pytest.mark.parametrize("bits,batch,window", [(2048, 41, 5), (2046, 37, 4), (1500, 29, 3), (4096, 9, 6),
                                               (3500, 7, 5), (1024, 70, 4), (3072, 13, 5), (512, 90, 4),
                                               (300, 33, 3)])
@pytest.mark.parametrize("layout", [IM, IL])
def test_truncated_karatsuba_modexp(mp, bits, batch, window, layout):
    """Exponentiation whose every product is in the truncated Karatsuba form (lazy when
    4N <= W^NP, i.e. 2046 and 1500 bits here), through both allocation paths."""
    b = _tkara_batch(bits, batch, 8300 + bits)
    ctx = mp.MontCtx(dev(mp, b.N, layout), batch, bits, layout)
    want = oracle.modexp(b.a, b.e, b.ebits, b.N)
    Y = out_tensor(mp, batch, b.n, layout)
    A, E = dev(mp, b.a, layout), dev(mp, b.e, layout)
    mp.modexp_consttime(Y, A, E, b.ebits, ctx, window, mp.RED_TRUNCATED, mp.ALGO_KARATSUBA)
    assert_equal(host(mp, Y, batch, b.n, layout), want, f"tkara modexp {bits}")
    Y.zero_()
    mp.modexp_consttime_noalloc(Y, A, E, b.ebits, ctx, window, mp.RED_TRUNCATED, mp.ALGO_KARATSUBA)
    assert_equal(host(mp, Y, batch, b.n, layout), want, f"tkara modexp noalloc {bits}")
    ctx.free()


@pytest.mark.parametrize("bits,windows", [(1000, (2, 4, 5)), (1024, (1, 4, 5)), (2048, (2, 3, 4)),
                                          (3072, (2, 3)), (4096, (1, 2))])
def test_modexp_shared_tables(mp, bits, windows):
    """Window tables in shared memory (mp_tune_set_table): equal to the oracle at every window
    whose tables fit, on the extremes and a ragged batch; at w = 6, where they do not fit, the
    call keeps the global tables and stays exact; the classical reduction keeps global tables."""
    batch = 45 if bits > 3000 else 77
    b = _tkara_batch(bits, batch, 8700 + bits)
    ctx = mp.MontCtx(dev(mp, b.N, IL), batch, bits, IL)
    want = oracle.modexp(b.a, b.e, b.ebits, b.N)
    A, E = dev(mp, b.a, IL), dev(mp, b.e, IL)
    Y = out_tensor(mp, batch, b.n, IL)
    assert mp.tune_get_table(bits) == mp.TABLE_GLOBAL
    try:
        mp.tune_set_table(bits, mp.TABLE_SHARED)
        assert mp.tune_get_table(bits) == mp.TABLE_SHARED
        for w in windows:
            assert mp.table_residency(bits, w) >= 32
            Y.zero_()
            mp.modexp_consttime(Y, A, E, b.ebits, ctx, w, mp.RED_TRUNCATED)
            assert_equal(host(mp, Y, batch, b.n, IL), want, f"shared tables {bits} w={w}")
        assert mp.table_residency(bits, 6) == 0
        for w, red in ((6, mp.RED_TRUNCATED), (windows[0], mp.RED_FULL)):
            Y.zero_()
            mp.modexp_consttime(Y, A, E, b.ebits, ctx, w, red)
            assert_equal(host(mp, Y, batch, b.n, IL), want, f"global fallback {bits} w={w} red={red}")
    finally:
        mp.tune_set_table(bits, mp.TABLE_GLOBAL)
    ctx.free()


@pytest.mark.parametrize("shape", [(16, 8), (8, 16)])
def test_modexp_each_4096_bit_shape(mp, shape):
    """Montgomery products and exponentiations on each role-swapped shape of the 4096-bit class,
    both block-product reductions, against the oracle (extremes, ragged batch)."""
    bits, batch = 4096, 37
    b = _tkara_batch(bits, batch, 8800)
    saved = mp.tune_get(bits)
    try:
        mp.tune_set(bits, *shape)
        ctx = mp.MontCtx(dev(mp, b.N, IL), batch, bits, IL)
        A, B, E = dev(mp, b.a, IL), dev(mp, b.b, IL), dev(mp, b.e, IL)
        C = out_tensor(mp, batch, b.n, IL)
        for red in (mp.RED_TRUNCATED, mp.RED_FULL):
            mp.mont_mul(C, A, B, ctx, red)
            assert_equal(host(mp, C, batch, b.n, IL), oracle.mont_def(b.a, b.b, b.N), f"mont_mul {shape} {red}")
            mp.modexp_consttime(C, A, E, b.ebits, ctx, 5, red)
            assert_equal(host(mp, C, batch, b.n, IL), oracle.modexp(b.a, b.e, b.ebits, b.N), f"modexp {shape} {red}")
        ctx.free()
    finally:
        mp.tune_set(bits, saved["G"], saved["M"], saved["window"], saved["karatsuba_from_bits"])


def test_truncated_karatsuba_unavailable(mp):
    """The Karatsuba form exists for the truncated reduction of the classes from 512 to 4096
    bits; the 256- and 4608-bit classes and the other reductions report MP_ERR_UNIMPLEMENTED
    before any work."""
    for bits, red in ((256, 0), (100, 0), (4108, 0), (4608, 0), (2048, 1), (2048, 2), (4096, 1), (1024, 2)):
        b = si.make_batch(0, "test", 4, bits, ebits=8, sub=8500 + bits + red)
        ctx = mp.MontCtx(dev(mp, b.N, IL), 4, bits, IL)
        C = out_tensor(mp, 4, b.n, IL)
        with pytest.raises(mp.MpError) as e:
            mp.mont_mul(C, dev(mp, b.a, IL), dev(mp, b.b, IL), ctx, red, mp.ALGO_KARATSUBA)
        assert e.value.status == -7
        with pytest.raises(mp.MpError) as e:
            mp.modexp_consttime(C, dev(mp, b.a, IL), dev(mp, b.e, IL), 8, ctx, 4, red, mp.ALGO_KARATSUBA)
        assert e.value.status == -7
        ctx.free()


# ------------------------------------------------------------------ mixed sizes in one call

def _mixed_jobs(mp, specs, layout):
    jobs, batches, outs = [], [], []
    for bits, batch, ebits, window, sub in specs:
        b = si.make_batch(0, "mixed", batch, bits, ebits=ebits, sub=sub)
        ctx = mp.MontCtx(dev(mp, b.N, layout), batch, bits, layout)
        Y = out_tensor(mp, batch, b.n, layout)
        jobs.append((Y, dev(mp, b.a, layout), dev(mp, b.e, layout), ebits, ctx, window))
        batches.append(b)
        outs.append(Y)
    return jobs, batches, outs


@pytest.mark.parametrize("layout", [IM, IL])
def test_mixed_matches_per_size(mp, layout):
    """Every job of a mixed call (all size classes, ragged batches, short exponents) equals
    modexp_consttime on that job alone, and sampled instances equal the oracle."""
    specs = [(2048, 70, 2048, 5, 1), (1024, 133, 1024, 4, 2), (3072, 21, 3072, 5, 3), (4096, 17, 4096, 6, 4),
             (512, 40, 300, 3, 5), (1000, 9, 64, 0, 6), (4108, 5, 128, 4, 7), (4607, 3, 96, 5, 8)]
    jobs, batches, outs = _mixed_jobs(mp, specs, layout)
    ws = mp.mixed_workspace(jobs)
    for red in (0, 1, 2):
        for Y in outs:
            Y.zero_()
        mp.modexp_consttime_mixed(jobs, red, ws)
        torch.cuda.synchronize()
        for (Y, A, E, ebits, ctx, window), b in zip(jobs, batches):
            Z = torch.zeros_like(Y)
            mp.modexp_consttime(Z, A, E, ebits, ctx, window, red)
            got = host(mp, Y, b.batch, b.n, layout)
            assert_equal(got, host(mp, Z, b.batch, b.n, layout), f"mixed vs one-size {b.bits} red={red}")
            idx = np.arange(0, b.batch, max(1, b.batch // 5))
            want = oracle.modexp(b.a[idx], b.e[idx], ebits, b.N[idx])
            assert_equal(got[idx], want, f"mixed vs oracle {b.bits} red={red}")


def test_mixed_routed_own_base_jobs(mp):
    """Requests routed to the instances of a context (a pool of moduli) with their own bases:
    each request's table is built per request; repeated and ragged entries; beside a
    fixed-base job on resident tables of the same context."""
    bits, pool, w = 2048, 10, 5
    b = si.make_batch(0, "mixed", pool, bits, ebits=1, sub=40)
    ctx = mp.MontCtx(dev(mp, b.N, IL), pool, bits, IL)
    tables = torch.empty(mp.modexp_table_bytes(ctx, w) // 4, dtype=torch.int32, device="cuda")
    mp.modexp_table_build(tables, dev(mp, b.a, IL), ctx, w)
    rng = si.stream(0, "test", "other", 41)
    for nreq in (1, 37):
        idx = rng.integers(0, pool, size=nreq).astype(np.uint32)
        base = si.uniform_below(rng, b.N[idx], bits)
        e = si.random_bits(rng, nreq, 300)
        Y1, Y2 = out_tensor(mp, nreq, b.n, IL), out_tensor(mp, nreq, b.n, IL)
        d_idx, d_e = mp.to_device(idx), dev(mp, e, IL)
        jobs = [(Y1, dev(mp, base, IL), d_e, 300, ctx, w, d_idx, None, nreq),
                (Y2, None, d_e, 300, ctx, w, d_idx, tables, nreq)]
        for red in (0, 1, 2):
            mp.modexp_consttime_mixed(jobs, red, mp.mixed_workspace(jobs))
            torch.cuda.synchronize()
            assert_equal(host(mp, Y1, nreq, b.n, IL), oracle.modexp(base, e, 300, b.N[idx]), f"own bases, red={red}")
            assert_equal(host(mp, Y2, nreq, b.n, IL), oracle.modexp(b.a[idx], e, 300, b.N[idx]), f"fixed, red={red}")
    ctx.free()


def test_mixed_many_jobs_and_limits(mp):
    """16 jobs (more than the call's parallel streams) in one call, twice in a row; a 17th job
    is rejected before any launch."""
    specs = [((1024, 2048, 512, 3072)[i % 4], 5 + i, 64, 0, 20 + i) for i in range(16)]
    jobs, batches, outs = _mixed_jobs(mp, specs, IL)
    ws = mp.mixed_workspace(jobs)
    for _ in range(2):
        for Y in outs:
            Y.zero_()
        mp.modexp_consttime_mixed(jobs, 0, ws)
        torch.cuda.synchronize()
        for (Y, A, E, ebits, ctx, window), b in zip(jobs, batches):
            want = oracle.modexp(b.a, b.e, ebits, b.N)
            assert_equal(host(mp, Y, b.batch, b.n, IL), want, f"16-job call, {b.bits} bits")
    with pytest.raises(mp.MpError) as e:
        mp.modexp_consttime_mixed(jobs + jobs[:1], 0, ws)
    assert e.value.status == -2


def test_tuning_round_trip(mp):
    for bits in (1024, 2048, 3072, 4096):
        cands = mp.shape_candidates(bits)
        assert len(cands) >= 1
        before = mp.tune_get(bits)
        for G, M in cands:
            mp.tune_set(bits, G, M, 4)
            t = mp.tune_get(bits)
            assert (t["G"], t["M"], t["window"]) == (G, M, 4)
            # results do not depend on the shape
            b = si.make_batch(0, "test", 12, bits, ebits=96, sub=bits + G)
            ctx = mp.MontCtx(dev(mp, b.N, IL), 12, bits, IL)
            Y = out_tensor(mp, 12, b.n, IL)
            mp.modexp_consttime(Y, dev(mp, b.a, IL), dev(mp, b.e, IL), 96, ctx, 0)
            assert_equal(host(mp, Y, 12, b.n, IL), oracle.modexp(b.a, b.e, 96, b.N), f"shape {G}x{M}")
            C = out_tensor(mp, 12, b.n, IL)
            mp.mont_mul(C, dev(mp, b.a, IL), dev(mp, b.b, IL), ctx)
            assert_equal(host(mp, C, 12, b.n, IL), oracle.mont_def(b.a, b.b, b.N), f"mont shape {G}x{M}")
        mp.tune_set(bits, before["G"], before["M"], 0)


@pytest.mark.parametrize("layout", [IM, IL])
def test_warp_mapped_shape(mp, layout):
    """The 2048-bit class's warp-mapped shape (thread t of every instance in warp t of a block,
    the lane is the instance): every entry point, several blocks plus a ragged one, extreme
    operands, all reductions (CIOS runs on a lane-mapped shape of the class)."""
    bits, batch = 2048, 77
    cands = mp.shape_candidates(bits)
    assert (-8, 8) in cands
    before = mp.tune_get(bits)
    mp.tune_set(bits, -8, 8, 5)
    try:
        b = si.make_batch(0, "test", batch, bits, sub=4242)
        b.a[3] = b.N[3] - np.array([1] + [0] * (b.n - 1), np.uint32)       # N-1
        b.a[4] = 0
        b.e[5] = 0
        n = b.n
        A, Bv, E = dev(mp, b.a, layout), dev(mp, b.b, layout), dev(mp, b.e, layout)
        C2 = torch.zeros(mp.array_words(layout, batch, 2 * n), dtype=torch.int32, device="cuda")
        mp.mp_mul(C2, A, Bv, batch, bits, layout, mp.ALGO_SCHOOLBOOK)
        assert_equal(host(mp, C2, batch, 2 * n, layout), oracle.mul(b.a, b.b), "mp_mul")
        mp.mp_sqr(C2, A, batch, bits, layout, mp.ALGO_SCHOOLBOOK)
        assert_equal(host(mp, C2, batch, 2 * n, layout), oracle.sqr(b.a), "mp_sqr")
        ctx = mp.MontCtx(dev(mp, b.N, layout), batch, bits, layout)
        C = out_tensor(mp, batch, n, layout)
        want_mul, want_sqr = oracle.mont_def(b.a, b.b, b.N), oracle.mont_def(b.a, b.a, b.N)
        want_exp = oracle.modexp(b.a, b.e, bits, b.N)
        for red in (0, 1, 2):
            mp.mont_mul(C, A, Bv, ctx, red)
            assert_equal(host(mp, C, batch, n, layout), want_mul, f"mont_mul red={red}")
            mp.mont_sqr(C, A, ctx, red)
            assert_equal(host(mp, C, batch, n, layout), want_sqr, f"mont_sqr red={red}")
            Y = out_tensor(mp, batch, n, layout)
            mp.modexp_consttime(Y, A, E, bits, ctx, 5, red)
            assert_equal(host(mp, Y, batch, n, layout), want_exp, f"modexp red={red}")
        if layout == IL:
            tables = torch.empty(mp.modexp_table_bytes(ctx, 5) // 4, dtype=torch.int32, device="cuda")
            mp.modexp_table_build(tables, A, ctx, 5)
            index = np.arange(batch, dtype=np.uint32)[::-1].copy()
            Y = out_tensor(mp, batch, n, IL)
            mp.modexp_fixed_base(Y, mp.to_device(index), dev(mp, b.e[index], IL), bits, batch, ctx, tables, 5)
            assert_equal(host(mp, Y, batch, n, IL), want_exp[index], "fixed base")
        ctx.free()
    finally:
        mp.tune_set(bits, before["G"], before["M"], 0)


@pytest.mark.parametrize("bits", [3100, 4000, 4096, 4108, 4154, 4608])
@pytest.mark.parametrize("layout", [IM, IL])
def test_two_level_karatsuba(mp, bits, layout):
    """Two levels of Karatsuba (9 quarter products) against the oracle, with operands that
    make every half and quarter sum carry (all ones) next to random ones."""
    batch = 45
    b = si.make_batch(0, "test", batch, bits, ebits=1, sub=6000 + bits)
    n = b.n
    top = np.uint32((1 << (bits - 32 * (n - 1))) - 1) if bits % 32 else np.uint32(0xFFFFFFFF)
    b.a[0, :] = 0xFFFFFFFF
    b.a[0, -1] = top
    b.b[0] = b.a[0]
    b.a[1] = 0
    A, B = dev(mp, b.a, layout), dev(mp, b.b, layout)
    C = torch.zeros(mp.array_words(layout, batch, 2 * n), dtype=torch.int32, device="cuda")
    mp.mp_mul(C, A, B, batch, bits, layout, mp.ALGO_KARATSUBA2)
    assert_equal(host(mp, C, batch, 2 * n, layout), oracle.mul(b.a, b.b), f"karatsuba2 mul {bits}")
    mp.mp_sqr(C, A, batch, bits, layout, mp.ALGO_KARATSUBA2)
    assert_equal(host(mp, C, batch, 2 * n, layout), oracle.sqr(b.a), f"karatsuba2 sqr {bits}")


def test_two_level_karatsuba_unavailable_sizes(mp):
    b = si.make_batch(0, "test", 4, 2048, ebits=1, sub=77)
    A = dev(mp, b.a, IL)
    C = torch.zeros(mp.array_words(IL, 4, 2 * b.n), dtype=torch.int32, device="cuda")
    with pytest.raises(mp.MpError) as e:
        mp.mp_mul(C, A, A, 4, 2048, IL, mp.ALGO_KARATSUBA2)
    assert e.value.status == -7


BOUNDARY_SIZES = [2, 3, 31, 32, 33, 63, 65, 255, 256, 257, 511, 513, 1023, 1025, 2047, 2049,
                  3071, 3073, 4095, 4097, 4607, 4608]


@pytest.mark.parametrize("bits", BOUNDARY_SIZES)
def test_size_class_boundaries(mp, bits):
    """Every size-class edge (one word less / more than a padded size, the smallest and the
    largest sizes): products, all three reductions, and a short exponentiation, on a ragged batch."""
    batch = 33
    b = si.make_batch(0, "test", batch, bits, ebits=min(bits, 96), sub=8000 + bits)
    n = b.n
    A, B = dev(mp, b.a, IL), dev(mp, b.b, IL)
    C2 = torch.zeros(mp.array_words(IL, batch, 2 * n), dtype=torch.int32, device="cuda")
    mp.mp_mul(C2, A, B, batch, bits, IL)
    assert_equal(host(mp, C2, batch, 2 * n, IL), oracle.mul(b.a, b.b), f"mp_mul {bits}")
    mp.mp_sqr(C2, A, batch, bits, IL)
    assert_equal(host(mp, C2, batch, 2 * n, IL), oracle.sqr(b.a), f"mp_sqr {bits}")
    ctx = mp.MontCtx(dev(mp, b.N, IL), batch, bits, IL)
    C = out_tensor(mp, batch, n, IL)
    want_mul, want_sqr = oracle.mont_def(b.a, b.b, b.N), oracle.mont_def(b.a, b.a, b.N)
    want_exp = oracle.modexp(b.a, b.e, b.ebits, b.N)
    for red in (0, 1, 2):
        mp.mont_mul(C, A, B, ctx, red)
        assert_equal(host(mp, C, batch, n, IL), want_mul, f"mont_mul {bits} red={red}")
        mp.mont_sqr(C, A, ctx, red)
        assert_equal(host(mp, C, batch, n, IL), want_sqr, f"mont_sqr {bits} red={red}")
        mp.modexp_consttime(C, A, dev(mp, b.e, IL), b.ebits, ctx, 3, red)
        assert_equal(host(mp, C, batch, n, IL), want_exp, f"modexp {bits} red={red}")
    ctx.free()


def test_bits_above_the_largest_class_are_rejected(mp):
    b = si.make_batch(0, "test", 2, 4608, ebits=1, sub=4609)
    with pytest.raises(mp.MpError):
        mp.MontCtx(dev(mp, np.concatenate([b.N, np.ones((2, 1), np.uint32)], axis=1), IL), 2, 4609, IL)


# ------------------------------------------------------------------ resident tables, fixed bases

@pytest.mark.parametrize("bits,window", [(1024, 4), (2048, 5), (3072, 5), (4096, 6)])
def test_fixed_base_requests(mp, bits, window):
    pool = 37
    b = si.make_batch(0, "serving", pool, bits, ebits=1, sub=bits)
    ctx = mp.MontCtx(dev(mp, b.N, IL), pool, bits, IL)
    tables = torch.empty(mp.modexp_table_bytes(ctx, window) // 4, dtype=torch.int32, device="cuda")
    mp.modexp_table_build(tables, dev(mp, b.a, IL), ctx, window)
    r = si.stream(0, "serving", "other", bits)
    nreq = 101
    index = r.integers(0, pool, nreq).astype(np.uint32)
    index[:3] = [0, pool - 1, 5]
    ebits = bits
    e = si.random_bits(si.stream(0, "serving", "exponent", bits), nreq, ebits)
    e[0] = 0
    Y = out_tensor(mp, nreq, b.n, IL)
    idx_t = mp.to_device(index)
    mp.modexp_fixed_base(Y, idx_t, dev(mp, e, IL), ebits, nreq, ctx, tables, window)
    got = host(mp, Y, nreq, b.n, IL)
    want = oracle.modexp(b.a[index], e, ebits, b.N[index])
    assert_equal(got, want, f"fixed base {bits}")
    # the same requests inside a mixed launch, next to an ordinary job
    b2 = si.make_batch(0, "serving", 19, 1024, sub=bits + 1)
    ctx2 = mp.MontCtx(dev(mp, b2.N, IL), 19, 1024, IL)
    Y2 = out_tensor(mp, 19, b2.n, IL)
    Y3 = out_tensor(mp, nreq, b.n, IL)
    jobs = [(Y3, None, dev(mp, e, IL), ebits, ctx, window, idx_t, tables, nreq),
            (Y2, dev(mp, b2.a, IL), dev(mp, b2.e, IL), 1024, ctx2, 4)]
    mp.modexp_consttime_mixed(jobs, 0, mp.mixed_workspace(jobs))
    assert_equal(host(mp, Y3, nreq, b.n, IL), want, "fixed base in a mixed launch")
    for red in (mp.RED_FULL, mp.RED_CIOS):   # the other reductions in the same launch
        Y3.zero_()
        Y2.zero_()
        mp.modexp_consttime_mixed(jobs, red, mp.mixed_workspace(jobs))
        assert_equal(host(mp, Y3, nreq, b.n, IL), want, f"fixed base in a mixed launch, red={red}")
        assert_equal(host(mp, Y2, 19, b2.n, IL), oracle.modexp(b2.a, b2.e, 1024, b2.N), f"ordinary job, red={red}")
    assert_equal(host(mp, Y2, 19, b2.n, IL), oracle.modexp(b2.a, b2.e, 1024, b2.N), "ordinary job beside it")


