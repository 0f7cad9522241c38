"""The autotuner times the library's kernels, returns a choice per size, and the choice
applied through mp_tune_set keeps results bit-exact."""
import pytest

import oracle
import seeded_inputs as si

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_tuner_small_run_and_apply():
    import paper_2410_18129_gb300 as mp
    from paper_2410_18129_gb300 import tune
    before = {b: mp.tune_get(b) for b in (1024, 2048)}
    choice = tune.tune(sizes=(1024, 2048), windows=(4, 5), rounds=1)
    assert set(choice) == {"1024", "2048"}
    for bits, c in choice.items():
        assert (c["G"], c["M"]) in mp.shape_candidates(int(bits))
        assert c["window"] in (4, 5) and c["modexp_per_s"] > 0 and c["table"] in ("global", "shared")
        assert all(r > 0 for r in c["residency_per_sm"].values())
    tune.apply(choice)
    for bits in (1024, 2048):
        t = mp.tune_get(bits)
        assert (t["G"], t["M"], t["window"]) == (choice[str(bits)]["G"], choice[str(bits)]["M"],
                                                  choice[str(bits)]["window"])
        b = si.make_batch(0, "test", 16, bits, ebits=200, sub=bits + 11)
        IL = mp.LAYOUT_INTERLEAVED
        dev = lambda x: mp.to_device(mp.interleave(x))
        ctx = mp.MontCtx(dev(b.N), 16, bits, IL)
        Y = torch.zeros(mp.array_words(IL, 16, b.n), dtype=torch.int32, device="cuda")
        mp.modexp_consttime(Y, dev(b.a), dev(b.e), 200, ctx, 0)
        got = mp.deinterleave(mp.to_host(Y), 16, b.n)
        assert (got == oracle.modexp(b.a, b.e, 200, b.N)).all()
    for b, t in before.items():
        mp.tune_set(b, t["G"], t["M"], 0, 0)
        mp.tune_set_table(b, mp.TABLE_GLOBAL)


def test_residency_and_montgomery_karatsuba_switch():
    """mp_shape_residency reports the kernels' occupancy; with the Montgomery switch-over set,
    AUTO exponentiations run the truncated Karatsuba form and still equal the oracle and the
    explicit MP_ALGO_KARATSUBA call."""
    import paper_2410_18129_gb300 as mp
    IL = mp.LAYOUT_INTERLEAVED
    for bits in (1024, 2048, 3072, 4096):
        for G, M in mp.shape_candidates(bits):
            assert mp.shape_residency(bits, G, M) > 0
        assert mp.shape_residency(bits, algo=mp.ALGO_KARATSUBA) > 0
    with pytest.raises(mp.MpError):
        mp.shape_residency(2048, 3, 3)                       # not a shape of the class
    bits = 2048
    b = si.make_batch(0, "test", 40, bits, ebits=300, sub=777)
    dev = lambda x: mp.to_device(mp.interleave(x))
    ctx = mp.MontCtx(dev(b.N), 40, bits, IL)
    A, E = dev(b.a), dev(b.e)
    Y_auto, Y_tk = (torch.zeros(mp.array_words(IL, 40, b.n), dtype=torch.int32, device="cuda") for _ in range(2))
    assert mp.tune_get_mont_karatsuba(bits) == 0
    try:
        mp.tune_set_mont_karatsuba(bits, 1025)
        assert mp.tune_get_mont_karatsuba(bits) == 1025
        mp.modexp_consttime(Y_auto, A, E, 300, ctx, 5)
        mp.modexp_consttime(Y_tk, A, E, 300, ctx, 5, mp.RED_TRUNCATED, mp.ALGO_KARATSUBA)
        torch.cuda.synchronize()
        got = mp.deinterleave(mp.to_host(Y_auto), 40, b.n)
        assert (got == oracle.modexp(b.a, b.e, 300, b.N)).all()
        assert torch.equal(Y_auto, Y_tk)
    finally:
        mp.tune_set_mont_karatsuba(bits, 0)
    ctx.free()
