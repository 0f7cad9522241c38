"""Property-based pins of the oracle's truncated reductions (Alg. 6 with Thm. 1 and Thm. 2,
and its Karatsuba form of Sec. 5.1): for moduli and T built from runs of all-ones and zero
words (the patterns that make every carry and borrow ripple) and random words, the recovered
high half equals floor(q*N / R) and the result equals T * R^-1 mod N, computed with Python's
integers."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")

W = 1 << 32
WORD = st.one_of(st.just(0), st.just(W - 1), st.just(1), st.just(W >> 1), st.integers(0, W - 1))


def words_value(ws):
    return sum(int(w) << (32 * i) for i, w in enumerate(ws))


@st.composite
def case(draw):
    n = draw(st.sampled_from([2, 4, 6, 8, 16]))
    R = 1 << (32 * n)
    N = words_value(draw(st.lists(WORD, min_size=n, max_size=n))) | 1 | (1 << (32 * n - 1))
    T = words_value(draw(st.lists(WORD, min_size=2 * n, max_size=2 * n))) % (N * R)
    return n, N, T


@hyp.settings(max_examples=300, deadline=None, derandomize=True)
@hyp.given(case())
def test_truncated_reductions_match_integers(c):
    n, N, T = c
    R = 1 << (32 * n)
    Np = (-pow(N, -1, R)) % R
    Nw, Npw, Tw = si.from_int(N, n), si.from_int(Np, n), si.from_int(T, 2 * n)
    q = (T % R) * Np % R
    want_H = q * N // R
    want_C = T * pow(R, -1, N) % N
    d6 = oracle.montred_alg6(Tw, Nw, Npw)
    assert si.to_int(d6["H"]) == want_H
    assert si.to_int(d6["C"]) == want_C
    dk = oracle.montred_tkara(Tw, Nw, Npw)
    assert si.to_int(dk["H"]) == want_H
    assert si.to_int(dk["C"]) == want_C
    assert abs(dk["e"]) <= n + 2          # 2h + 2 with h = n/2
    assert si.to_int(dk["Cpre"]) == (T + q * N) // R < 2 * N
