"""The stored fixture tests/golden/modexp_small.txt (written by make_fixtures.py from the
oracle): every value is re-derived from Python's own integers (pow, modular inverse), which
share nothing with the oracle, and the oracle must still reproduce it. The GPU test runs the
same instances through the C ABI."""
import os

import numpy as np
import pytest

import oracle
import seeded_inputs as si

HERE = os.path.dirname(os.path.abspath(__file__))


def rows():
    out = []
    with open(os.path.join(HERE, "golden", "modexp_small.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            bits, w, N, a, e, y, m = line.split()
            out.append((int(bits), int(w), int(N, 16), int(a, 16), int(e, 16), int(y, 16), int(m, 16)))
    return out


def test_fixture_against_python_integers():
    rs = rows()
    assert len(rs) == 9
    for bits, w, N, a, e, y, m in rs:
        n = (bits + 31) // 32
        assert N % 2 == 1 and N >> (bits - 1) == 1 and a < N
        assert y == pow(a, e, N)
        R = 1 << (32 * n)
        assert m == a * a * pow(R, -1, N) % N


def test_oracle_reproduces_fixture():
    for bits, w, N, a, e, y, m in rows():
        n = (bits + 31) // 32
        Nw, aw, ew = (si.from_ints([v], n) for v in (N, a, e))
        assert si.to_int(oracle.modexp(aw, ew, bits, Nw)[0]) == y
        assert si.to_int(oracle.mont_def(aw, aw, Nw)[0]) == m


@pytest.mark.gpu
def test_gpu_reproduces_fixture():
    torch = pytest.importorskip("torch")
    import paper_2410_18129_gb300 as mp
    for bits in sorted({r[0] for r in rows()}):
        rs = [r for r in rows() if r[0] == bits]
        n = (bits + 31) // 32
        N, a, e = (si.from_ints([r[k] for r in rs], n) for k in (2, 3, 4))
        B = len(rs)
        ctx = mp.MontCtx(mp.to_device(N.reshape(-1)), B, bits, mp.LAYOUT_INSTANCE_MAJOR)
        Y = torch.zeros(B * n, dtype=torch.int32, device="cuda")
        forms = [(mp.RED_TRUNCATED, mp.ALGO_AUTO), (mp.RED_FULL, mp.ALGO_AUTO), (mp.RED_CIOS, mp.ALGO_AUTO)]
        if bits > 256:   # the truncated Karatsuba form exists from the 512-bit class up
            forms.append((mp.RED_TRUNCATED, mp.ALGO_KARATSUBA))
        for red, algo in forms:
            mp.modexp_consttime(Y, mp.to_device(a.reshape(-1)), mp.to_device(e.reshape(-1)), bits, ctx, 5, red, algo)
            got = mp.to_host(Y).reshape(B, n)
            assert [si.to_int(v) for v in got] == [r[5] for r in rs], (bits, red, algo)
            mp.mont_mul(Y, mp.to_device(a.reshape(-1)), mp.to_device(a.reshape(-1)), ctx, red, algo)
            got = mp.to_host(Y).reshape(B, n)
            assert [si.to_int(v) for v in got] == [r[6] for r in rs], (bits, red, algo)
        ctx.free()
