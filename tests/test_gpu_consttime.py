"""Constant time of the exponentiation (Alg. 7: every window costs w squarings and one
product over a masked scan of the whole table, whatever the exponent and base), tested
dudect-style: per-instance SM cycle counts (modexp_timing_probe) of a fixed class of
secret inputs against a class of random inputs, in alternating runs of 64 instances of the
same launches (whole blocks of either kernel mapping), compared with Welch's t-test.
|t| < 4.5 is the usual pass threshold. A positive control shows that the same statistic
flags a 2 % timing difference at the same threshold: the public exponent length, 1024
against 1004 bits (measured t of about 6 with 512 run medians per class)."""
import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

BITS, W, BATCH, RUN, LAUNCHES = 1024, 5, 16384, 64, 4
IL = 1


def welch_t(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float((a.mean() - b.mean()) / np.sqrt(a.var(ddof=1) / a.size + b.var(ddof=1) / b.size))


@pytest.fixture(scope="module")
def setup():
    import paper_2410_18129_gb300 as mp
    b = si.make_batch(0, "test", BATCH, BITS, sub=4242)
    dev = lambda x: mp.to_device(mp.interleave(x))
    ctx = mp.MontCtx(dev(b.N), BATCH, BITS, IL)
    ws = torch.empty(mp.modexp_workspace_bytes(BATCH, BITS, W) // 4, dtype=torch.int32, device="cuda")
    yield mp, b, dev, ctx, ws
    ctx.free()


def run_samples(mp, ctx, ws, A, E, ebits, red):
    """Median cycles of each run of RUN instances, over LAUNCHES launches: [launches, runs]."""
    n = (BITS + 31) // 32
    y = torch.zeros(mp.array_words(IL, BATCH, n), dtype=torch.int32, device="cuda")
    cyc = torch.zeros(2 * BATCH, dtype=torch.int32, device="cuda")   # 64-bit counts
    mp.modexp_timing_probe(cyc, y, A, E, ebits, ctx, W, red, ws)   # warm-up
    out = []
    for _ in range(LAUNCHES):
        mp.modexp_timing_probe(cyc, y, A, E, ebits, ctx, W, red, ws)
        torch.cuda.synchronize()
        c = cyc.view(torch.int64).cpu().numpy().reshape(-1, RUN)
        assert (c > 0).all()
        out.append(np.median(c, axis=1))
    return np.stack(out)


SPECIAL = ["e=0", "e=all ones", "a=0", "a=1", "a=N-1"]


@pytest.mark.parametrize("red", [0, 2])
@pytest.mark.parametrize("case", SPECIAL)
def test_secret_inputs_do_not_change_cycles(setup, case, red):
    mp, b, dev, ctx, ws = setup
    n = b.n
    a, e = b.a.copy(), b.e.copy()
    fixed = (np.arange(BATCH) // RUN) % 2 == 0          # alternating runs: fixed class, random class
    if case == "e=0":
        e[fixed] = 0
    elif case == "e=all ones":
        e[fixed] = 0xFFFFFFFF
    elif case == "a=0":
        a[fixed] = 0
    elif case == "a=1":
        a[fixed] = 0
        a[fixed, 0] = 1
    else:
        a[fixed] = b.N[fixed]
        a[fixed, 0] -= np.uint32(1)                       # N odd: N-1 without borrow
    s = run_samples(mp, ctx, ws, dev(a), dev(e), BITS, red)
    t = welch_t(s[:, 0::2].ravel(), s[:, 1::2].ravel())
    print(f"{case}, red={red}: t = {t:.2f}")
    assert abs(t) < 4.5, f"{case}, red={red}: t = {t:.2f}"


def test_the_statistic_sees_a_two_percent_difference(setup):
    """Positive control on public data: 1024- against 1004-bit exponents (201 windows
    instead of 205) in alternating launches."""
    mp, b, dev, ctx, ws = setup
    A, E = dev(b.a), dev(b.e)
    long_, short = [], []
    for _ in range(4):
        long_.append(run_samples(mp, ctx, ws, A, E, 1024, 0))
        short.append(run_samples(mp, ctx, ws, A, E, 1004, 0))
    t = welch_t(np.concatenate(long_).ravel(), np.concatenate(short).ravel())
    print(f"control: t = {t:.2f}")
    assert t > 4.5, f"t = {t:.2f}: the statistic misses a 2 % difference"
