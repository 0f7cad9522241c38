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
    choice = tune.tune(sizes=(1024, 2048), windows=(4, 5), batch=1024)
    assert set(choice) == {"1024", "2048"}
    for bits, c in choice.items():
        assert (c["G"], c["M"]) in mp.shape_candidates(int(bits))
        assert c["window"] in (4, 5) and c["modexp_per_s"] > 0
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
